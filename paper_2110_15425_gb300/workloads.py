"""Seeded synthetic inputs for the five workloads (numpy only).

This module holds no model arithmetic: it only draws the per-trial parameters,
weights, conditions and positions that both the CUDA library and the CPU
oracle take as inputs. The paper's PsyNeuLink models and data are not
available, so these inputs stand in for them with the shapes, sizes and value
ranges of the workloads described in Sec. 2.1 and Sec. 5 (Botvinick Stroop,
DDM/LCA integrators, Predator-Prey, Multitasking):

- ``stroop_small``: colour/word/task inputs (2 each, one-hot) -> hidden colour,
  hidden word (logistic, bias -4) -> response (2); weights U[-2.5, 2.5];
  4 conditions x 1,000 trials.
- ``ddm``: drift A ~ U[0.1, 1], threshold z ~ U[0.5, 2] per trial.
- ``lca``: inputs I_i ~ U[0, 1] per trial and accumulator.
- ``predator_prey``: player/predator/prey positions U[-10, 10]^2 per trial,
  30 attention levels in [0, 1] per entity.
- ``stroop_wide``: stimulus one-hot 16 + task one-hot 16 -> hidden 256 ->
  response 16 (the wide multitask network).

Model noise is not drawn here: each side generates it from its own
Philox4x32-10 keyed by (seed, trial, candidate, step).
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _u(rng, lo, hi, shape):
    return rng.uniform(lo, hi, size=shape).astype(F32)


# --------------------------------------------------------------- Stroop ---

STROOP_LAYERS = [
    dict(name="color", size=2, input=True),
    dict(name="word", size=2, input=True),
    dict(name="task", size=2, input=True),
    dict(name="hidden_color", size=2, input=False, gain=1.0, bias=-4.0),
    dict(name="hidden_word", size=2, input=False, gain=1.0, bias=-4.0),
    dict(name="response", size=2, input=False, gain=1.0, bias=0.0),
]
# (sender, receiver) in projection-id order
STROOP_EDGES = [(0, 3), (1, 4), (2, 3), (2, 4), (3, 5), (4, 5)]


def stroop_conditions() -> np.ndarray:
    """4 conditions: k>>1 = task (0 colour naming, 1 word reading),
    k&1 = incongruent word. Row = [colour(2), word(2), task(2)]."""
    rows = []
    for k in range(4):
        task = [1.0, 0.0] if (k >> 1) == 0 else [0.0, 1.0]
        color = [1.0, 0.0]
        word = [1.0, 0.0] if (k & 1) == 0 else [0.0, 1.0]
        rows.append(color + word + task)
    return np.array(rows, dtype=F32)


def stroop_small(weight_seed: int = 0, noise_seed: int = 1, trials_per_condition: int = 1000,
                 weight_range: float = 2.5, max_steps: int = 500):
    rng = _rng(weight_seed)
    projections = []
    for s, r in STROOP_EDGES:
        W = _u(rng, -weight_range, weight_range,
               (STROOP_LAYERS[r]["size"], STROOP_LAYERS[s]["size"]))
        projections.append((s, r, W))
    return dict(layers=[dict(l) for l in STROOP_LAYERS], projections=projections,
                cond_inputs=stroop_conditions(), cond_block=trials_per_condition,
                n_trials=4 * trials_per_condition, rate=0.1, noise_sd=0.01,
                stop_layer=5, stop_threshold=0.7, max_steps=max_steps, seed=noise_seed)


# ----------------------------------------------------------- wide Stroop ---

WIDE_STIM = 16
WIDE_TASK = 16
WIDE_HIDDEN = 256
WIDE_RESP = 16


def stroop_wide(weight_seed: int = 4, noise_seed: int = 5, n_trials: int = 65536,
                hidden_range: float = 6.0, resp_range: float = 2.0, resp_bias: float = -8.0,
                max_steps: int = 500, hidden: int = WIDE_HIDDEN):
    """Wide multitask network. Trial t: stimulus t % 16, task (t // 16) % 16,
    i.e. condition t % 256 with condition c = task*16 + stim.

    The paper gives no sizes or weights for this network; hidden weights
    U[-6, 6], response weights U[-2, 2] and response bias -8 make about a
    quarter of the trials reach the stop criterion early (10-20 steps) while
    the rest run to the 500-step cap, so trial lengths are uneven."""
    rng = _rng(weight_seed)
    layers = [
        dict(name="stimulus", size=WIDE_STIM, input=True),
        dict(name="task", size=WIDE_TASK, input=True),
        dict(name="hidden", size=hidden, input=False, gain=1.0, bias=-4.0),
        dict(name="response", size=WIDE_RESP, input=False, gain=1.0, bias=resp_bias),
    ]
    projections = [
        (0, 2, _u(rng, -hidden_range, hidden_range, (hidden, WIDE_STIM))),
        (1, 2, _u(rng, -hidden_range, hidden_range, (hidden, WIDE_TASK))),
        (2, 3, _u(rng, -resp_range, resp_range, (WIDE_RESP, hidden))),
    ]
    cond = np.zeros((WIDE_STIM * WIDE_TASK, WIDE_STIM + WIDE_TASK), F32)
    for c in range(WIDE_STIM * WIDE_TASK):
        cond[c, c % WIDE_STIM] = 1.0
        cond[c, WIDE_STIM + c // WIDE_STIM] = 1.0
    return dict(layers=layers, projections=projections, cond_inputs=cond, cond_block=1,
                n_trials=n_trials, rate=0.1, noise_sd=0.01, stop_layer=3,
                stop_threshold=0.7, max_steps=max_steps, seed=noise_seed)


# ------------------------------------------------------------------ DDM ---

def ddm(n_trials: int = 1 << 20, param_seed: int = 1, noise_seed: int = 11):
    rng = _rng(param_seed)
    A = _u(rng, 0.1, 1.0, n_trials)
    z = _u(rng, 0.5, 2.0, n_trials)
    return dict(A=A, z=z, dt=1e-3, sigma=1.0, x0=0.0, max_steps=10000, seed=noise_seed)


# ------------------------------------------------------------------ LCA ---

def lca(n_trials: int = 262144, N: int = 8, input_seed: int = 2, noise_seed: int = 12):
    rng = _rng(input_seed + 1000 * N)
    I = _u(rng, 0.0, 1.0, (n_trials, N))
    return dict(I=I, N=N, leak=0.2, inhibition=0.3, sigma=0.1, dt=0.01, threshold=1.0,
                max_steps=3000, seed=noise_seed)


# -------------------------------------------------------- predator-prey ---

def predator_prey(n_trials: int = 64, levels: int = 30, pos_seed: int = 3, noise_seed: int = 13):
    rng = _rng(pos_seed)
    pos = _u(rng, -10.0, 10.0, (n_trials, 6))
    lv = (np.arange(levels, dtype=np.float64) / (levels - 1)).astype(F32)
    return dict(pos=pos, levels=[lv.copy(), lv.copy(), lv.copy()], obs_offset=0.1,
                pred_weight=0.5, seed=noise_seed)


def predator_prey_episodes(n_episodes: int = 64, levels: int = 30, n_trials: int = 64,
                           max_steps: int = 100, pos_seed: int = 21, noise_seed: int = 23):
    """Start positions of time-stepped episodes: player, predator and prey
    uniform on [-10, 10]^2; the same allocation levels as the grid search.
    Player steps 1.0, predator 0.6, prey 0.5 per time step; capture radius 1."""
    rng = _rng(pos_seed)
    start = _u(rng, -10.0, 10.0, (n_episodes, 6))
    lv = (np.arange(levels, dtype=np.float64) / (levels - 1)).astype(F32)
    return dict(start=start, levels=[lv.copy(), lv.copy(), lv.copy()], n_trials=n_trials,
                max_steps=max_steps, obs_offset=0.1, pred_weight=0.5, speed=(1.0, 0.6, 0.5),
                radius=1.0, seed=noise_seed)


def extended_stroop(weight_seed: int = 0, noise_seed: int = 1, trials_per_condition: int = 1000):
    """Extended Stroop (Sec. 5): the Stroop network plus two DDM nodes on its
    response layer, colour naming and finger pointing, with drifts
    W [2][2] . y_response + 0.2, dt 1e-3, sigma 1, bound 1, at most 10,000 steps."""
    w = stroop_small(weight_seed=weight_seed, noise_seed=noise_seed,
                     trials_per_condition=trials_per_condition)
    w["ddm_W"] = np.array([[2.0, -2.0], [-1.5, 1.5]], F32)
    w["ddm_bias"] = 0.2
    w["ddm_dt"] = 1e-3
    w["ddm_sigma"] = 1.0
    w["ddm_bound"] = 1.0
    w["ddm_max"] = 10000
    return w
