"""FP64 CPU oracle for the cognitive-model hot path (arXiv 2110.15425).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users. The CUDA library never
imports, links or calls anything here, and nothing here touches the CUDA
library.

The C sources (``rng.c``, ``models.c``) are compiled with gcc into
``oracle/_build/liboracle.so`` with ``-ffp-contract=off`` so that every
expression is evaluated as written. This module is a ctypes shim that turns
numpy arrays into pointers; ctypes releases the GIL during each call, so
several Python threads can run the oracle on disjoint trials at once (the
multicore layout of Sec. 3.6: each thread takes a segment of the work).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["rng.c", "models.c"]
_lock = threading.Lock()
_lib = None

MAX_LAYERS = 16
MAX_PROJ = 32


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no vector intrinsics)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_SO):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(_SO) >= newest:
            return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
    return _lib


class OrNet(C.Structure):
    _fields_ = [
        ("n_layers", C.c_int),
        ("size", C.c_int * MAX_LAYERS),
        ("is_input", C.c_int * MAX_LAYERS),
        ("gain", C.c_double * MAX_LAYERS),
        ("bias", C.c_double * MAX_LAYERS),
        ("rate", C.c_double),
        ("noise_sd", C.c_double),
        ("n_proj", C.c_int),
        ("proj_sender", C.c_int * MAX_PROJ),
        ("proj_receiver", C.c_int * MAX_PROJ),
        ("proj_w", C.c_void_p * MAX_PROJ),
        ("stop_layer", C.c_int),
        ("stop_threshold", C.c_double),
        ("max_steps", C.c_int32),
    ]


def _bind(L):
    P = C.c_void_p
    L.or_philox4x32_10.argtypes = [P, P, P]
    L.or_philox_words.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                  C.c_int64, P]
    L.or_uniform.argtypes = [C.c_uint32]
    L.or_uniform.restype = C.c_double
    L.or_weights.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_double, C.c_double, P]
    L.or_box_muller.argtypes = [P, P]
    L.or_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_int64, P]
    L.or_ddm_run.argtypes = [P, P, P, C.c_int64, C.c_uint64, C.c_double, C.c_double, C.c_double,
                             C.c_int32, P, P, P, P]
    L.or_lca_run.argtypes = [C.c_int, P, P, C.c_int64, C.c_uint64, C.c_double, C.c_double,
                             C.c_double, C.c_double, C.c_double, C.c_int32, C.c_int, C.c_int,
                             P, P, P, P]
    L.or_transfer_run.argtypes = [C.POINTER(OrNet), P, C.c_int, C.c_int, P, C.c_int64,
                                  C.c_uint64, P, P, P, P, P, C.c_int32]
    L.or_pp_outcome.argtypes = [P, P, C.c_uint64, C.c_uint32, C.c_uint32, C.c_double,
                                C.c_double, P]
    L.or_pp_outcome.restype = C.c_double
    L.or_pp_means.argtypes = [P, C.c_int32, P, C.c_int32, P, C.c_int32, P, C.c_int32, P,
                              C.c_int64, C.c_uint64, C.c_double, C.c_double, P]
    L.or_argmax.argtypes = [P, C.c_int64, P, P, P]
    L.or_ddm_run_offset.argtypes = [P, P, C.c_int64, C.c_uint32, C.c_uint64, C.c_double,
                                    C.c_double, C.c_double, C.c_int32, P, P, P, P]
    L.or_argmax_reservoir.argtypes = [P, C.c_int64, C.c_uint64, P, P, P, P]
    L.or_extended_run.argtypes = [C.POINTER(OrNet), P, C.c_int, C.c_int, P, C.c_int64,
                                  C.c_uint64, C.c_int, P, P, P, P, P, P, P, P, P, P, P, P, P,
                                  P, P, P, P]
    L.or_pp_episode.argtypes = [P, C.c_uint32, P, C.c_int32, P, C.c_int32, P, C.c_int32,
                                C.c_int32, C.c_int32, C.c_uint64, C.c_double, C.c_double, P,
                                C.c_double, P, P, P, P, P, P, P, P]
    L.or_pp_refine.argtypes = [P, C.c_int32, P, P, C.c_int32, C.c_int32, C.c_uint64, C.c_double,
                               C.c_double, P, P, P, P, P]
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _ids(trial_ids, n):
    if trial_ids is None:
        return np.arange(n, dtype=np.uint32)
    return _c(trial_ids, np.uint32)


def _threaded(fn, n, threads):
    """Run fn(lo, hi) on `threads` contiguous segments of range(n)."""
    threads = max(1, min(int(threads), n if n > 0 else 1))
    if threads == 1:
        fn(0, n)
        return
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)
    ts = [threading.Thread(target=fn, args=(int(bounds[i]), int(bounds[i + 1])))
          for i in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()


# ------------------------------------------------------------------ RNG ---

def philox(ctr, key):
    """One Philox4x32-10 block for ctr[4], key[2] (uint32)."""
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def philox_words(seed, trial, cand, purpose, block0, nblocks):
    out = np.zeros(4 * nblocks, np.uint32)
    lib().or_philox_words(seed, trial, cand, purpose, block0, nblocks, _p(out))
    return out


def uniform(w):
    return lib().or_uniform(int(w))


def weights(seed, proj, n, lo, hi):
    """Seeded weights of projection `proj`: n float32 values in [lo, hi]."""
    out = np.zeros(n, np.float32)
    lib().or_weights(seed, proj, n, lo, hi, _p(out))
    return out


def box_muller(words):
    w = _c(words, np.uint32)
    z = np.zeros(4, np.float64)
    lib().or_box_muller(_p(w), _p(z))
    return z


def normals(seed, trial, cand, d0, n):
    out = np.zeros(n, np.float64)
    lib().or_normals(seed, trial, cand, d0, n, _p(out))
    return out


# ------------------------------------------------------------------ DDM ---

def ddm_run(A, z, seed, dt=1e-3, sigma=1.0, x0=0.0, max_steps=10000, trial_ids=None,
            threads=1):
    """Returns dict(choice int8, step int32, x double, margin double) per id."""
    A = _c(A, np.float32)
    z = _c(z, np.float32)
    ids = _ids(trial_ids, A.shape[0])
    n = ids.shape[0]
    out = dict(choice=np.zeros(n, np.int8), step=np.zeros(n, np.int32),
               x=np.zeros(n, np.float64), margin=np.zeros(n, np.float64))
    L = lib()

    def run(lo, hi):
        if hi <= lo:
            return
        L.or_ddm_run(_p(A), _p(z), _p(ids[lo:]), hi - lo, seed, dt, sigma, x0, max_steps,
                     _p(out["choice"][lo:]), _p(out["step"][lo:]), _p(out["x"][lo:]),
                     _p(out["margin"][lo:]))
    _threaded(run, n, threads)
    return out


def ddm_run_offset(A, z, seed, trial0, dt=1e-3, sigma=1.0, x0=0.0, max_steps=10000):
    """DDM trials of a run starting at global id trial0 (trial k: A[k], z[k],
    noise of id trial0 + k)."""
    A = _c(A, np.float32)
    z = _c(z, np.float32)
    n = A.shape[0]
    out = dict(choice=np.zeros(n, np.int8), step=np.zeros(n, np.int32),
               x=np.zeros(n, np.float64), margin=np.zeros(n, np.float64))
    lib().or_ddm_run_offset(_p(A), _p(z), n, trial0, seed, dt, sigma, x0, max_steps,
                            _p(out["choice"]), _p(out["step"]), _p(out["x"]), _p(out["margin"]))
    return out


# ------------------------------------------------------------------ LCA ---

def lca_run(I, seed, leak=0.2, inhibition=0.3, sigma=0.1, dt=0.01, threshold=1.0,
            max_steps=3000, rectify=True, two_sided=False, trial_ids=None, threads=1):
    I = _c(I, np.float32)
    ntr, N = I.shape
    ids = _ids(trial_ids, ntr)
    n = ids.shape[0]
    out = dict(choice=np.zeros(n, np.int8), step=np.zeros(n, np.int32),
               x=np.zeros((n, N), np.float64), margin=np.zeros(n, np.float64))
    L = lib()

    def run(lo, hi):
        if hi <= lo:
            return
        L.or_lca_run(N, _p(I), _p(ids[lo:]), hi - lo, seed, leak, inhibition, sigma, dt,
                     threshold, max_steps, int(rectify), int(two_sided),
                     _p(out["choice"][lo:]), _p(out["step"][lo:]), _p(out["x"][lo:]),
                     _p(out["margin"][lo:]))
    _threaded(run, n, threads)
    return out


# ------------------------------------------------------- transfer network ---

def _net(layers, projections, rate, noise_sd, stop_layer, stop_threshold, max_steps):
    """layers: list of dict(size, input: bool, gain, bias);
    projections: list of (sender, receiver, W[recv][send] float32)."""
    net = OrNet()
    net.n_layers = len(layers)
    for i, l in enumerate(layers):
        net.size[i] = int(l["size"])
        net.is_input[i] = 1 if l.get("input", False) else 0
        net.gain[i] = float(l.get("gain", 1.0))
        net.bias[i] = float(l.get("bias", 0.0))
    net.rate = rate
    net.noise_sd = noise_sd
    net.n_proj = len(projections)
    keep = []
    for p, (s, r, W) in enumerate(projections):
        W = _c(W, np.float32)
        assert W.shape == (layers[r]["size"], layers[s]["size"])
        keep.append(W)
        net.proj_sender[p] = s
        net.proj_receiver[p] = r
        net.proj_w[p] = W.ctypes.data
    net.stop_layer = stop_layer
    net.stop_threshold = stop_threshold
    net.max_steps = max_steps
    return net, keep


def transfer_run(layers, projections, cond_inputs, cond_block, seed, rate=0.1, noise_sd=0.01,
                 stop_layer=None, stop_threshold=0.7, max_steps=500, trial_ids=None,
                 n_trials=None, trace_steps=0, threads=1):
    if stop_layer is None:
        stop_layer = len(layers) - 1
    net, keep = _net(layers, projections, rate, noise_sd, stop_layer, stop_threshold, max_steps)
    cin = _c(cond_inputs, np.float32)
    n_cond = cin.shape[0]
    ids = _ids(trial_ids, n_trials if n_trials is not None else n_cond * cond_block)
    n = ids.shape[0]
    ssize = layers[stop_layer]["size"]
    total = sum(l["size"] for l in layers)
    out = dict(choice=np.zeros(n, np.int8), step=np.zeros(n, np.int32),
               y=np.zeros((n, ssize), np.float64), margin=np.zeros(n, np.float64))
    if trace_steps:
        out["trace"] = np.zeros((n, trace_steps + 1, total), np.float64)
    L = lib()

    def run(lo, hi):
        if hi <= lo:
            return
        tr = _p(out["trace"][lo:]) if trace_steps else None
        L.or_transfer_run(C.byref(net), _p(cin), n_cond, cond_block, _p(ids[lo:]), hi - lo,
                          seed, _p(out["choice"][lo:]), _p(out["step"][lo:]),
                          _p(out["y"][lo:]), _p(out["margin"][lo:]), tr, trace_steps)
    _threaded(run, n, threads)
    del keep
    return out


def extended_run(layers, projections, cond_inputs, cond_block, seed, ddm_W, ddm_bias, ddm_dt,
                 ddm_sigma, ddm_bound, ddm_max, rate=0.1, noise_sd=0.01, stop_layer=None,
                 stop_threshold=0.7, max_steps=500, trial_ids=None, n_trials=None, threads=1):
    """Extended Stroop (Sec. 5): the network, then DDM nodes driven by its
    response layer. ddm_W [n_ddm][stop size], per-DDM bias, dt, sigma, bound,
    max steps."""
    if stop_layer is None:
        stop_layer = len(layers) - 1
    net, keep = _net(layers, projections, rate, noise_sd, stop_layer, stop_threshold, max_steps)
    cin = _c(cond_inputs, np.float32)
    n_cond = cin.shape[0]
    ids = _ids(trial_ids, n_trials if n_trials is not None else n_cond * cond_block)
    n = ids.shape[0]
    W = _c(ddm_W, np.float32)
    q = W.shape[0]
    ss = layers[stop_layer]["size"]
    assert W.shape == (q, ss)
    b = _c(ddm_bias, np.float32)
    dt, sg, bd = (_c(v, np.float64) for v in (ddm_dt, ddm_sigma, ddm_bound))
    mx = _c(ddm_max, np.int32)
    out = dict(choice=np.zeros(n, np.int8), step=np.zeros(n, np.int32),
               s_choice=np.zeros(n, np.int8), s_step=np.zeros(n, np.int32),
               y=np.zeros((n, ss)), s_margin=np.zeros(n), drift=np.zeros((n, q)),
               d_choice=np.zeros((n, q), np.int8), d_step=np.zeros((n, q), np.int32),
               d_x=np.zeros((n, q)), d_margin=np.zeros((n, q)))
    L = lib()

    def run(lo, hi):
        if hi <= lo:
            return
        L.or_extended_run(C.byref(net), _p(cin), n_cond, cond_block, _p(ids[lo:]), hi - lo, seed,
                          q, _p(W), _p(b), _p(dt), _p(sg), _p(bd), _p(mx),
                          *[_p(out[k][lo:]) for k in ("choice", "step", "s_choice", "s_step", "y",
                                                      "s_margin", "drift", "d_choice", "d_step",
                                                      "d_x", "d_margin")])
    _threaded(run, n, threads)
    del keep
    return out


# ------------------------------------------------------ predator-prey grid ---

def pp_outcome(pos, a, seed, trial, cand, obs_offset=0.1, pred_weight=0.5):
    pos = _c(pos, np.float32)
    a = _c(a, np.float64)
    per = np.zeros(6, np.float64)
    v = lib().or_pp_outcome(_p(pos), _p(a), seed, trial, cand, obs_offset, pred_weight,
                            _p(per))
    return v, per


def pp_means(pos, levels, seed, cand_ids=None, obs_offset=0.1, pred_weight=0.5, threads=1):
    """levels: three float32 arrays (player, predator, prey)."""
    pos = _c(pos, np.float32)
    lv = [_c(l, np.float32) for l in levels]
    n_c = lv[0].shape[0] * lv[1].shape[0] * lv[2].shape[0]
    ids = _ids(cand_ids, n_c)
    n = ids.shape[0]
    means = np.zeros(n, np.float64)
    L = lib()

    def run(lo, hi):
        if hi <= lo:
            return
        L.or_pp_means(_p(pos), pos.shape[0], _p(lv[0]), lv[0].shape[0], _p(lv[1]),
                      lv[1].shape[0], _p(lv[2]), lv[2].shape[0], _p(ids[lo:]), hi - lo, seed,
                      obs_offset, pred_weight, _p(means[lo:]))
    _threaded(run, n, threads)
    return means


def argmax(v):
    v = _c(v, np.float64)
    b = C.c_int64()
    bv = C.c_double()
    g = C.c_double()
    lib().or_argmax(_p(v), v.shape[0], C.byref(b), C.byref(bv), C.byref(g))
    return int(b.value), float(bv.value), float(g.value)


def argmax_reservoir(v, seed):
    """(best index, best value, gap, number of ties): random choice among exact
    ties by reservoir sampling (Sec. 3.3)."""
    v = _c(v, np.float64)
    b = C.c_int64()
    bv = C.c_double()
    g = C.c_double()
    k = C.c_int64()
    lib().or_argmax_reservoir(_p(v), v.shape[0], seed, C.byref(b), C.byref(bv), C.byref(g),
                              C.byref(k))
    return int(b.value), float(bv.value), float(g.value), int(k.value)


def pp_refine(pos, lo, hi, points, rounds, seed, obs_offset=0.1, pred_weight=0.5):
    """Coarse-to-fine grid search (Sec. 4.3 by simulation): per round the best
    index, its mean, the runner-up gap, the round's box (lo[3], hi[3]) and the
    best allocation."""
    pos = _c(pos, np.float32)
    lo = _c(lo, np.float32)
    hi = _c(hi, np.float32)
    best = np.zeros(rounds, np.int64)
    value = np.zeros(rounds, np.float64)
    gap = np.zeros(rounds, np.float64)
    box = np.zeros((rounds, 6), np.float32)
    alloc = np.zeros((rounds, 3), np.float32)
    lib().or_pp_refine(_p(pos), pos.shape[0], _p(lo), _p(hi), points, rounds, seed, obs_offset,
                       pred_weight, _p(best), _p(value), _p(gap), _p(box), _p(alloc))
    return dict(best=best, value=value, gap=gap, box=box, alloc=alloc)


def pp_episodes(start, levels, n_trials, max_steps, seed, episode_ids=None, obs_offset=0.1,
                pred_weight=0.5, speed=(1.0, 0.6, 0.5), radius=1.0, threads=1):
    """Time-stepped predator-prey episodes (Sec. 2.1), one per row of start
    [E][6] (episode id = row, or episode_ids). Returns outcome, steps, final
    positions and per-step trajectories (best index, its mean, gap, positions,
    capture margin; -1 / nan after the end)."""
    start = _c(start, np.float32)
    lv = [_c(l, np.float32) for l in levels]
    E = start.shape[0]
    ids = np.arange(E, dtype=np.uint32) if episode_ids is None else _c(episode_ids, np.uint32)
    sp = _c(speed, np.float64)
    outc = np.zeros(E, np.int8)
    steps = np.zeros(E, np.int32)
    fin = np.zeros((E, 6), np.float32)
    best = np.full((E, max_steps), -1, np.int64)
    gap = np.full((E, max_steps), np.nan)
    val = np.full((E, max_steps), np.nan)
    pos = np.full((E, max_steps, 6), np.nan, np.float32)
    marg = np.full((E, max_steps), np.nan)
    L = lib()

    def run(lo, hi):
        for k in range(lo, hi):
            o = C.c_int8()
            s = C.c_int32()
            L.or_pp_episode(_p(start[k]), int(ids[k]), _p(lv[0]), lv[0].shape[0], _p(lv[1]),
                            lv[1].shape[0], _p(lv[2]), lv[2].shape[0], n_trials, max_steps, seed,
                            obs_offset, pred_weight, _p(sp), radius, C.byref(o), C.byref(s),
                            _p(fin[k]), _p(best[k]), _p(val[k]), _p(gap[k]), _p(pos[k]),
                            _p(marg[k]))
            outc[k] = o.value
            steps[k] = s.value
    _threaded(run, E, threads)
    return dict(outcome=outc, steps=steps, final=fin, best=best, value=val, gap=gap, pos=pos,
                margin=marg)
