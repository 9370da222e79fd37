"""ctypes binding of the C ABI declared in include/distill_gpu.h.

Argument marshalling only: every step of the hot path runs in the CUDA
library. There is no fallback: if ``_lib/libdistill_gpu.so`` is missing the
import of ``lib()`` raises. Device buffers are torch CUDA tensors (PyTorch is
used for device memory and streams only); their ``data_ptr()`` values are
passed as plain device pointers.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdistill_gpu.so")

DG_OK, DG_E_ARG, DG_E_SHAPE, DG_E_BUDGET, DG_E_CUDA, DG_E_TIMEOUT, DG_E_UNSUPPORTED, DG_E_STATE = (
    0, -1, -2, -3, -4, -5, -6, -7)
STATUS_NAMES = {0: "DG_OK", -1: "DG_E_ARG", -2: "DG_E_SHAPE", -3: "DG_E_BUDGET", -4: "DG_E_CUDA",
                -5: "DG_E_TIMEOUT", -6: "DG_E_UNSUPPORTED", -7: "DG_E_STATE"}

DG_INPUT, DG_TRANSFER_LOGISTIC, DG_DDM, DG_LCA, DG_PP_OBSERVE, DG_PP_ACTION, DG_PP_OBJECTIVE = range(7)
DG_LCA_NO_RECTIFY, DG_LCA_TWO_SIDED = 1, 2
DG_F32, DG_BF16 = 0, 1
DG_MODE_BATCHED, DG_MODE_PLAIN = 0, 1
DG_TIE_LOWEST, DG_TIE_RESERVOIR = 0, 1
MODEL_KINDS = {0: "ddm", 1: "lca", 2: "transfer", 3: "transfer_wide", 4: "predator_prey"}


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class dg_mechanism(C.Structure):
    _fields_ = [("kind", C.c_int32), ("size", C.c_int32), ("gain", C.c_double),
                ("bias", C.c_double), ("rate", C.c_double), ("noise", C.c_double),
                ("dt", C.c_double), ("leak", C.c_double), ("inhibition", C.c_double),
                ("start", C.c_double), ("offset", C.c_double), ("weight", C.c_double),
                ("flags", C.c_int32), ("reserved", C.c_int32), ("threshold", C.c_double),
                ("max_steps", C.c_int32), ("reserved2", C.c_int32)]


class dg_projection(C.Structure):
    _fields_ = [("sender", C.c_int32), ("receiver", C.c_int32), ("weights", C.c_void_p),
                ("dtype", C.c_int32), ("reserved", C.c_int32), ("lo", C.c_double),
                ("hi", C.c_double)]


class dg_stop(C.Structure):
    _fields_ = [("mech", C.c_int32), ("max_steps", C.c_int32), ("threshold", C.c_double)]


class dg_run_desc(C.Structure):
    _fields_ = [("n_trials", C.c_int64), ("trial_offset", C.c_int64), ("seed", C.c_uint64),
                ("trial_params", C.c_void_p),
                ("cond_inputs", C.c_void_p), ("n_cond", C.c_int32), ("cond_block", C.c_int32),
                ("mode", C.c_int32), ("reserved", C.c_int32)]


class dg_grid_desc(C.Structure):
    _fields_ = [("n_levels", C.c_int32 * 3), ("n_trials", C.c_int32),
                ("levels", C.c_void_p * 3), ("positions", C.c_void_p), ("seed", C.c_uint64),
                ("mode", C.c_int32), ("tie_break", C.c_int32), ("cand_begin", C.c_int64),
                ("cand_count", C.c_int64)]


class dg_episode_desc(C.Structure):
    _fields_ = [("n_episodes", C.c_int32), ("max_steps", C.c_int32),
                ("n_levels", C.c_int32 * 3), ("n_trials", C.c_int32),
                ("levels", C.c_void_p * 3), ("start", C.c_void_p), ("seed", C.c_uint64),
                ("speed", C.c_double * 3), ("capture_radius", C.c_double),
                ("episode_offset", C.c_int64)]


class dg_episode_out(C.Structure):
    _fields_ = [("outcome", C.c_void_p), ("steps", C.c_void_p), ("final_pos", C.c_void_p),
                ("best", C.c_void_p), ("value", C.c_void_p), ("pos", C.c_void_p)]


class dg_refine_desc(C.Structure):
    _fields_ = [("points", C.c_int32), ("rounds", C.c_int32), ("n_trials", C.c_int32),
                ("reserved", C.c_int32), ("lo", C.c_float * 3), ("hi", C.c_float * 3),
                ("positions", C.c_void_p), ("seed", C.c_uint64)]


class dg_refine_round(C.Structure):
    _fields_ = [("alloc", C.c_float * 3), ("lo", C.c_float * 3), ("hi", C.c_float * 3),
                ("round", C.c_int32), ("best_index", C.c_int64), ("best_value", C.c_double),
                ("runner_up_gap", C.c_double)]


class dg_grid_result(C.Structure):
    _fields_ = [("best_index", C.c_int64), ("best_value", C.c_double),
                ("runner_up_gap", C.c_double)]


class dg_job(C.Structure):
    _fields_ = [("model", C.c_void_p), ("is_grid", C.c_int32), ("reserved", C.c_int32),
                ("run", dg_run_desc), ("grid", dg_grid_desc), ("choice", C.c_void_p),
                ("step", C.c_void_p), ("final_state", C.c_void_p),
                ("grid_result", C.c_void_p), ("cand_means", C.c_void_p)]


class dg_job_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("reserved", C.c_int32), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("device_bytes", C.c_uint64)]


EXPORTS = [
    "dg_create", "dg_destroy", "dg_last_error", "dg_version", "dg_compose", "dg_model_free",
    "dg_model_info", "dg_run", "dg_grid_search", "dg_argmax_f64", "dg_philox_words",
    "dg_normals", "dg_batch_create", "dg_batch_add_run", "dg_batch_add_grid",
    "dg_batch_launch", "dg_batch_kernels", "dg_batch_free", "dg_submit", "dg_wait", "dg_serve_stats",
    "dg_grid_search_noalloc", "dg_stream_status", "dg_selftest_wait_timeout",
    "dg_argmax_f64_reservoir", "dg_grid_refine", "dg_run_episodes", "dg_selftest_pair_sum",
    "dg_grid_search_batch", "dg_model_weights", "dg_run_jobs", "dg_tune_stats",
]

_lib = None
_lock = threading.Lock()


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
            L = C.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    P, S = C.c_void_p, C.c_int
    i32, i64, u32, u64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
    sig = {
        "dg_create": [C.POINTER(P), S, C.c_size_t],
        "dg_destroy": [P],
        "dg_compose": [P, C.POINTER(dg_mechanism), i32, C.POINTER(dg_projection), i32,
                       C.POINTER(dg_stop), u64, C.POINTER(P)],
        "dg_model_weights": [P, i32, P, i64],
        "dg_model_free": [P],
        "dg_model_info": [P, C.POINTER(i32), C.POINTER(i32)],
        "dg_run": [P, C.POINTER(dg_run_desc), P, P, P, P],
        "dg_grid_search": [P, C.POINTER(dg_grid_desc), P, P, P],
        "dg_grid_search_noalloc": [P, C.POINTER(dg_grid_desc), P, P, P],
        "dg_grid_search_batch": [P, i32, C.POINTER(dg_grid_desc), P, P, P],
        "dg_run_jobs": [P, i32, C.POINTER(dg_run_desc), P, P, P, P],
        "dg_tune_stats": [P, P, P],
        "dg_stream_status": [P, P],
        "dg_selftest_wait_timeout": [P, i32, P],
        "dg_selftest_pair_sum": [P, i64, i32, i32, P, P],
        "dg_argmax_f64": [P, P, i64, P, P],
        "dg_argmax_f64_reservoir": [P, P, i64, u64, P, P],
        "dg_grid_refine": [P, C.POINTER(dg_refine_desc), P, P],
        "dg_run_episodes": [P, C.POINTER(dg_episode_desc), C.POINTER(dg_episode_out), P],
        "dg_philox_words": [u64, u32, u32, u32, u32, i64, P, P],
        "dg_normals": [u64, u32, u32, u64, i64, P, P],
        "dg_batch_create": [P, C.POINTER(P)],
        "dg_batch_add_run": [P, P, C.POINTER(dg_run_desc), P, P, P],
        "dg_batch_add_grid": [P, P, C.POINTER(dg_grid_desc), P, P],
        "dg_batch_launch": [P, P],
        "dg_batch_kernels": [P, P],
        "dg_batch_free": [P],
        "dg_submit": [P, C.POINTER(dg_job), C.POINTER(u64)],
        "dg_wait": [P, u64, i32, C.POINTER(dg_job_result)],
        "dg_serve_stats": [P, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(u64)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = S
    L.dg_last_error.restype = C.c_char_p
    L.dg_last_error.argtypes = []
    L.dg_version.restype = C.c_char_p
    L.dg_version.argtypes = []


def check(status):
    if status != DG_OK:
        raise DGError(status, lib().dg_last_error().decode())
    return status


def ptr(t):
    """Device (or host) address of a torch tensor / numpy array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t.ctypes.data)


def stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ------------------------------------------------------------ thin wrappers ---

def dg_create(device=0, hbm_budget_bytes=0):
    h = C.c_void_p()
    check(lib().dg_create(C.byref(h), device, hbm_budget_bytes))
    return h


def dg_destroy(ctx):
    check(lib().dg_destroy(ctx))


def dg_version():
    return lib().dg_version().decode()


def dg_last_error():
    return lib().dg_last_error().decode()


def dg_compose(ctx, mechs, projs, stop, weight_seed=0):
    m = (dg_mechanism * len(mechs))(*mechs)
    p = (dg_projection * max(1, len(projs)))(*projs) if projs else None
    out = C.c_void_p()
    check(lib().dg_compose(ctx, m, len(mechs), p, len(projs), C.byref(stop), weight_seed,
                           C.byref(out)))
    return out


def dg_model_weights(model, proj_index, n):
    """The FP32 weights the model holds for projection proj_index (n floats)."""
    import numpy as np
    out = np.zeros(max(n, 1), np.float32)
    check(lib().dg_model_weights(model, proj_index, out.ctypes.data_as(C.c_void_p), n))
    return out[:n]


def dg_model_free(model):
    check(lib().dg_model_free(model))


def dg_model_info(model):
    k, s = C.c_int32(), C.c_int32()
    check(lib().dg_model_info(model, C.byref(k), C.byref(s)))
    return k.value, s.value


def dg_run(model, desc, choice, step, final_state=None, stream=None):
    check(lib().dg_run(model, C.byref(desc), ptr(choice), ptr(step), ptr(final_state),
                       stream_handle(stream)))


def dg_tune_stats(ctx):
    """(tuned launch-shape keys, launches that ran an untuned default shape)."""
    a, b = C.c_int64(), C.c_int64()
    check(lib().dg_tune_stats(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def dg_run_jobs(model, descs, choices, steps, final_states=None, stream=None):
    """descs: list of dg_run_desc (device trial_params); choices, steps: lists
    of device tensors; final_states: list of device tensors (or None entries)
    or None."""
    n = len(descs)
    arr = (dg_run_desc * n)(*descs)
    ch = (C.c_void_p * n)(*[t.data_ptr() for t in choices])
    st = (C.c_void_p * n)(*[t.data_ptr() for t in steps])
    fs = None
    if final_states is not None:
        fs = (C.c_void_p * n)(*[None if t is None else t.data_ptr() for t in final_states])
    check(lib().dg_run_jobs(model, n, arr, ch, st, fs, stream_handle(stream)))


def dg_grid_search(model, desc, result, cand_means=None, stream=None):
    check(lib().dg_grid_search(model, C.byref(desc), ptr(result), ptr(cand_means),
                               stream_handle(stream)))


def dg_grid_search_batch(model, descs, results, cand_means=None, stream=None):
    """descs: list of dg_grid_desc; results: device tensor of len(descs) x 3
    doubles; cand_means: list of device tensors (or None entries) or None."""
    n = len(descs)
    arr = (dg_grid_desc * n)(*descs)
    means = None
    if cand_means is not None:
        means = (C.c_void_p * n)(*[None if t is None else t.data_ptr() for t in cand_means])
    check(lib().dg_grid_search_batch(model, n, arr, ptr(results), means, stream_handle(stream)))


def dg_grid_search_noalloc(model, desc, result, cand_means=None, stream=None):
    check(lib().dg_grid_search_noalloc(model, C.byref(desc), ptr(result), ptr(cand_means),
                                       stream_handle(stream)))


def dg_selftest_wait_timeout(ctx, wait_us, stream=None):
    check(lib().dg_selftest_wait_timeout(ctx, wait_us, stream_handle(stream)))


def dg_selftest_pair_sum(values, n_groups, per_group, lanes, means, stream=None):
    check(lib().dg_selftest_pair_sum(ptr(values), n_groups, per_group, lanes, ptr(means),
                                     stream_handle(stream)))


def dg_stream_status(ctx, stream=None):
    check(lib().dg_stream_status(ctx, stream_handle(stream)))


def dg_argmax_f64(ctx, values, result, stream=None):
    check(lib().dg_argmax_f64(ctx, ptr(values), values.numel(), ptr(result),
                              stream_handle(stream)))


def episode_desc(levels, start, n_trials, max_steps, seed, speed=(1.0, 0.6, 0.5), radius=1.0,
                 episode_offset=0):
    d = dg_episode_desc()
    d.episode_offset = episode_offset
    d._keep = (tuple(levels), start)
    d.n_episodes = start.shape[0]
    d.max_steps = max_steps
    d.n_trials = n_trials
    for i in range(3):
        d.n_levels[i] = levels[i].numel()
        d.levels[i] = levels[i].data_ptr()
        d.speed[i] = float(speed[i])
    d.start = start.data_ptr()
    d.seed = seed
    d.capture_radius = float(radius)
    return d


def episode_out(outcome, steps, final_pos=None, best=None, value=None, pos=None):
    o = dg_episode_out()
    o._keep = (outcome, steps, final_pos, best, value, pos)
    o.outcome, o.steps = ptr(outcome), ptr(steps)
    o.final_pos, o.best, o.value, o.pos = ptr(final_pos), ptr(best), ptr(value), ptr(pos)
    return o


def dg_run_episodes(model, desc, out, stream=None):
    check(lib().dg_run_episodes(model, C.byref(desc), C.byref(out), stream_handle(stream)))


def dg_grid_refine(model, desc, rounds, stream=None):
    """rounds: device uint8 tensor of desc.rounds * 64 bytes (dg_refine_round[])."""
    check(lib().dg_grid_refine(model, C.byref(desc), ptr(rounds), stream_handle(stream)))


def refine_desc(positions, lo, hi, points, rounds, seed):
    d = dg_refine_desc()
    d._keep = positions
    d.points = points
    d.rounds = rounds
    d.n_trials = positions.shape[0]
    for i in range(3):
        d.lo[i] = float(lo[i])
        d.hi[i] = float(hi[i])
    d.positions = positions.data_ptr()
    d.seed = seed
    return d


def refine_rounds(raw):
    """Decode dg_refine_round[] from host bytes into numpy arrays."""
    import numpy as np
    rec = np.dtype([("alloc", "<f4", 3), ("lo", "<f4", 3), ("hi", "<f4", 3), ("round", "<i4"),
                    ("best_index", "<i8"), ("best_value", "<f8"), ("runner_up_gap", "<f8")])
    assert rec.itemsize == C.sizeof(dg_refine_round) == 64
    return np.frombuffer(np.ascontiguousarray(raw).tobytes(), dtype=rec)


def dg_argmax_f64_reservoir(ctx, values, seed, result, stream=None):
    check(lib().dg_argmax_f64_reservoir(ctx, ptr(values), values.numel(), seed, ptr(result),
                                        stream_handle(stream)))


def dg_philox_words(seed, trial, cand, purpose, block0, nblocks, out, stream=None):
    check(lib().dg_philox_words(seed, trial, cand, purpose, block0, nblocks, ptr(out),
                                stream_handle(stream)))


def dg_normals(seed, trial, cand, d0, n, out, stream=None):
    check(lib().dg_normals(seed, trial, cand, d0, n, ptr(out), stream_handle(stream)))


def dg_batch_create(ctx):
    h = C.c_void_p()
    check(lib().dg_batch_create(ctx, C.byref(h)))
    return h


def dg_batch_add_run(batch, model, desc, choice, step, final_state=None):
    check(lib().dg_batch_add_run(batch, model, C.byref(desc), ptr(choice), ptr(step),
                                 ptr(final_state)))


def dg_batch_add_grid(batch, model, desc, result, cand_means=None):
    check(lib().dg_batch_add_grid(batch, model, C.byref(desc), ptr(result), ptr(cand_means)))


def dg_batch_launch(batch, stream=None):
    check(lib().dg_batch_launch(batch, stream_handle(stream)))


def dg_batch_kernels(batch):
    """Kernel launches one dg_batch_launch makes (after the first launch)."""
    n = C.c_int64(0)
    check(lib().dg_batch_kernels(batch, C.byref(n)))
    return n.value


def dg_batch_free(batch):
    check(lib().dg_batch_free(batch))


def dg_submit(ctx, job):
    t = C.c_uint64()
    check(lib().dg_submit(ctx, C.byref(job), C.byref(t)))
    return t.value


def dg_wait(ctx, ticket, timeout_ms=-1):
    r = dg_job_result()
    check(lib().dg_wait(ctx, ticket, timeout_ms, C.byref(r)))
    return r


def dg_serve_stats(ctx):
    q, r, d, b = C.c_int64(), C.c_int64(), C.c_int64(), C.c_uint64()
    check(lib().dg_serve_stats(ctx, C.byref(q), C.byref(r), C.byref(d), C.byref(b)))
    return dict(queued=q.value, running=r.value, done=d.value, bytes_in_use=b.value)


# ---------------------------------------------------- model graph builders ---

def mech(kind, size, **kw):
    m = dg_mechanism()
    m.kind = kind
    m.size = size
    m.gain = kw.get("gain", 1.0)
    for k, v in kw.items():
        setattr(m, k, v)
    return m


def proj(sender, receiver, weights=None, dtype=DG_F32, lo=0.0, hi=0.0):
    """weights: numpy float32 [recv][send] (kept alive by the caller until compose
    returns), or None with lo < hi for weights drawn from the compose seed."""
    p = dg_projection()
    p.sender = sender
    p.receiver = receiver
    p.weights = None if weights is None else weights.ctypes.data
    p.dtype = dtype
    p.lo = lo
    p.hi = hi
    return p


def stop(mech_index, max_steps, threshold=0.0):
    s = dg_stop()
    s.mech = mech_index
    s.max_steps = max_steps
    s.threshold = threshold
    return s


def compose_ddm(ctx, dt=1e-3, sigma=1.0, x0=0.0, max_steps=10000):
    return dg_compose(ctx, [mech(DG_DDM, 1, dt=dt, noise=sigma, start=x0)], [],
                      stop(0, max_steps))


def compose_lca(ctx, N, leak=0.2, inhibition=0.3, sigma=0.1, dt=0.01, threshold=1.0,
                max_steps=3000, rectify=True, two_sided=False):
    flags = (0 if rectify else DG_LCA_NO_RECTIFY) | (DG_LCA_TWO_SIDED if two_sided else 0)
    return dg_compose(ctx, [mech(DG_LCA, N, dt=dt, noise=sigma, leak=leak, inhibition=inhibition,
                                 flags=flags)], [], stop(0, max_steps, threshold))


def compose_network(ctx, layers, projections, rate=0.1, noise_sd=0.01, stop_layer=None,
                    stop_threshold=0.7, max_steps=500, bf16_edges=(), weight_seed=0):
    """layers: dicts (size, input, gain, bias); projections: (sender, receiver, W), W a
    [recv][send] array, or a (lo, hi) pair for weights drawn from weight_seed."""
    import numpy as np
    ms = []
    for l in layers:
        if l.get("input", False):
            ms.append(mech(DG_INPUT, int(l["size"])))
        else:
            ms.append(mech(DG_TRANSFER_LOGISTIC, int(l["size"]), gain=float(l.get("gain", 1.0)),
                           bias=float(l.get("bias", 0.0)), rate=rate, noise=noise_sd))
    ps, keep = [], []
    for i, (s, r, W) in enumerate(projections):
        dt = DG_BF16 if i in bf16_edges else DG_F32
        if isinstance(W, tuple):
            ps.append(proj(s, r, None, dt, lo=float(W[0]), hi=float(W[1])))
        else:
            keep.append(np.ascontiguousarray(W, dtype=np.float32))
            ps.append(proj(s, r, keep[-1], dt))
    if stop_layer is None:
        stop_layer = len(layers) - 1
    model = dg_compose(ctx, ms, ps, stop(stop_layer, max_steps, stop_threshold), weight_seed)
    del keep
    return model


def compose_extended_stroop(ctx, layers, projections, ddm_nodes, rate=0.1, noise_sd=0.01,
                            stop_layer=None, stop_threshold=0.7, max_steps=500):
    """The Stroop network plus DDM nodes on its stop layer (Sec. 5).
    ddm_nodes: list of mechanisms, each dict(W [units][stop size], bias, dt,
    sigma, bound, max_steps), appended after the layers in order; each is fed
    by one projection from the stop layer with weights W."""
    import numpy as np
    if stop_layer is None:
        stop_layer = len(layers) - 1
    ms = []
    for l in layers:
        if l.get("input", False):
            ms.append(mech(DG_INPUT, int(l["size"])))
        else:
            ms.append(mech(DG_TRANSFER_LOGISTIC, int(l["size"]), gain=float(l.get("gain", 1.0)),
                           bias=float(l.get("bias", 0.0)), rate=rate, noise=noise_sd))
    keep = [np.ascontiguousarray(W, dtype=np.float32) for (_, _, W) in projections]
    ps = [proj(s, r, keep[i]) for i, (s, r, _) in enumerate(projections)]
    for nd in ddm_nodes:
        W = np.ascontiguousarray(nd["W"], dtype=np.float32)
        keep.append(W)
        ms.append(mech(DG_DDM, W.shape[0], bias=float(nd.get("bias", 0.0)), dt=float(nd["dt"]),
                       noise=float(nd["sigma"]), threshold=float(nd["bound"]),
                       max_steps=int(nd["max_steps"])))
        ps.append(proj(stop_layer, len(ms) - 1, W))
    model = dg_compose(ctx, ms, ps, stop(stop_layer, max_steps, stop_threshold))
    del keep
    return model


def compose_predator_prey(ctx, obs_offset=0.1, pred_weight=0.5):
    ms = [mech(DG_INPUT, 6), mech(DG_PP_OBSERVE, 6, offset=obs_offset),
          mech(DG_PP_ACTION, 2, weight=pred_weight), mech(DG_PP_OBJECTIVE, 1)]
    ps = [proj(0, 1), proj(1, 2), proj(2, 3)]
    return dg_compose(ctx, ms, ps, stop(3, 1))


def run_desc(n_trials, seed, trial_params=None, cond_inputs=None, n_cond=0, cond_block=1,
             mode=DG_MODE_BATCHED, trial_offset=0):
    d = dg_run_desc()
    d.n_trials = n_trials
    d.trial_offset = trial_offset
    d.seed = seed
    d.trial_params = None if trial_params is None else trial_params.data_ptr()
    d.cond_inputs = None if cond_inputs is None else cond_inputs.data_ptr()
    # the struct holds raw addresses: keep the tensors alive as long as it lives
    d._keep = (trial_params, cond_inputs)
    d.n_cond = n_cond
    d.cond_block = cond_block
    d.mode = mode
    return d


def grid_desc(levels, positions, seed, mode=DG_MODE_BATCHED, cand_begin=0, cand_count=0,
              tie_break=DG_TIE_LOWEST):
    d = dg_grid_desc()
    d.tie_break = tie_break
    d._keep = (tuple(levels), positions)
    d.cand_begin = cand_begin
    d.cand_count = cand_count
    for i in range(3):
        d.n_levels[i] = levels[i].numel()
        d.levels[i] = levels[i].data_ptr()
    d.n_trials = positions.shape[0]
    d.positions = positions.data_ptr()
    d.seed = seed
    d.mode = mode
    return d
