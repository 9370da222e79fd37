"""Pins for the oracle's layered logistic network and predator-prey grid search.

Transfer network (Sec. 2.2, 3.3; Botvinick Stroop):
- noise-free time-averaging integrator with constant input has the closed
  form s(t) = net (1 - (1 - rate)^t), y = logistic(gain (s + bias));
- synchronous update (the current/previous output structures of Sec. 3.3):
  a change at a layer's input reaches the next layer one step later;
- logistic outputs lie in (0, 1) (Sec. 4.1);
- noise is added to the state: stationary variance sd^2 / (1 - (1 - rate)^2);
- the stop rule on closed-form trajectories.

Predator-prey (Sec. 2.1):
- noise-free geometric cases of the one-step move;
- perception noise sd = 1 / (offset + allocation);
- candidate index layout and cost-only ordering without perception noise;
- argmax with lowest-index ties.
"""
import math

import numpy as np
import pytest

from paper_2110_15425_gb300 import workloads as W


def _logistic(x):
    return 1.0 / (1.0 + math.exp(-x))


def _chain(w_in, w_out, bias_h=-4.0, bias_r=0.0):
    layers = [dict(size=1, input=True), dict(size=1, bias=bias_h), dict(size=2, bias=bias_r)]
    proj = [(0, 1, np.array([[w_in]], np.float32)),
            (1, 2, np.array([[w_out], [-w_out]], np.float32))]
    return layers, proj


def test_integrator_closed_form(orc):
    layers, proj = _chain(2.5, 1.0, bias_h=-1.0)
    o = orc.transfer_run(layers, proj, np.array([[1.0]], np.float32), 1, seed=0, noise_sd=0.0,
                         n_trials=1, trace_steps=200, stop_threshold=10.0)
    tr = o["trace"][0]
    w = float(np.float32(2.5))
    for t in range(201):
        s = w * (1 - 0.9**t)
        assert math.isclose(tr[t, 1], _logistic(s - 1.0), rel_tol=1e-12), t
    assert tr[0, 0] == 1.0 and np.all(tr[:, 0] == 1.0)  # clamped input


def test_initial_outputs(orc):
    w = W.stroop_small()
    o = orc.transfer_run(w["layers"], w["projections"], w["cond_inputs"], 1, seed=1, n_trials=4,
                         trace_steps=1)
    tr = o["trace"]
    h0 = 1.0 / (1.0 + math.exp(4.0))
    assert np.allclose(tr[:, 0, 6:10], h0, rtol=1e-15)     # hidden units
    assert np.allclose(tr[:, 0, 10:12], 0.5, rtol=1e-15)   # response, bias 0


def test_synchronous_delay(orc):
    """Response at step 1 reads the hidden outputs of step 0, which do not
    depend on the input weights; at step 2 they do."""
    a = orc.transfer_run(*_chain(3.0, 2.0), np.array([[1.0]], np.float32), 1, seed=0,
                         noise_sd=0.0, n_trials=1, trace_steps=3, stop_threshold=10.0)["trace"][0]
    b = orc.transfer_run(*_chain(-3.0, 2.0), np.array([[1.0]], np.float32), 1, seed=0,
                         noise_sd=0.0, n_trials=1, trace_steps=3, stop_threshold=10.0)["trace"][0]
    assert a[1, 1] != b[1, 1]                 # hidden moves at step 1
    assert np.array_equal(a[1, 2:], b[1, 2:])  # response does not yet
    assert not np.array_equal(a[2, 2:], b[2, 2:])


def test_logistic_range(orc):
    w = W.stroop_small(weight_seed=4, trials_per_condition=20)
    o = orc.transfer_run(w["layers"], w["projections"], w["cond_inputs"], 20, seed=3,
                         n_trials=80, trace_steps=100)
    tr = o["trace"][:, :, 6:]
    assert np.all(tr > 0.0) and np.all(tr < 1.0)


def test_noise_added_to_state(orc):
    """net = 0, bias 0: s(t) = 0.9 s(t-1) + sd eps_t, so Var s(t) =
    sd^2 (1 - 0.81^t) / 0.19; s is recovered from y by the logit."""
    layers = [dict(size=1, input=True), dict(size=1, bias=0.0)]
    proj = [(0, 1, np.array([[0.0]], np.float32))]
    n, T = 20000, 60
    o = orc.transfer_run(layers, proj, np.array([[1.0]], np.float32), 1, seed=21, noise_sd=0.01,
                         n_trials=n, trace_steps=T, stop_threshold=10.0, stop_layer=1)
    y = o["trace"][:, T, 1]
    s = np.log(y / (1 - y))
    var = 1e-4 * (1 - 0.81**T) / 0.19
    assert abs(s.var() / var - 1) < 5 * math.sqrt(2.0 / n)
    assert abs(s.mean()) < 5 * math.sqrt(var / n)
    # step 1: s(1) = sd * eps of noisy unit 0 at step 1 (normal 0)
    y1 = o["trace"][0, 1, 1]
    eps = orc.normals(21, 0, 0, 0, 1)[0]
    assert math.isclose(math.log(y1 / (1 - y1)), 0.01 * eps, rel_tol=1e-9)


def test_stop_rule_closed_form(orc):
    """Inputs straight into a 2-unit response, noise-free: s_i(t) = w_i (1 - 0.9^t);
    stop at the first t with |y0 - y1| > 0.7."""
    for w0, w1, first in [(3.0, -2.0, 0), (-1.0, 4.0, 1), (1.2, -1.1, None)]:
        layers = [dict(size=2, input=True), dict(size=2, bias=0.0)]
        proj = [(0, 1, np.array([[w0, 0.0], [0.0, w1]], np.float32))]
        o = orc.transfer_run(layers, proj, np.array([[1.0, 1.0]], np.float32), 1, seed=0,
                             noise_sd=0.0, n_trials=1, stop_layer=1, max_steps=500)
        f0, f1 = float(np.float32(w0)), float(np.float32(w1))
        tstar = None
        for t in range(1, 501):
            g = abs(_logistic(f0 * (1 - 0.9**t)) - _logistic(f1 * (1 - 0.9**t)))
            if g > 0.7:
                tstar = t
                break
        if first is None:
            assert tstar is None and o["choice"][0] == -1 and o["step"][0] == 500
        else:
            assert o["step"][0] == tstar and o["choice"][0] == first


def test_condition_mapping(orc):
    """Trial t takes condition (t // cond_block) % n_cond."""
    w = W.stroop_small(weight_seed=4, trials_per_condition=3)
    ids = np.arange(12, dtype=np.uint32)
    full = orc.transfer_run(w["layers"], w["projections"], w["cond_inputs"], 3, seed=2,
                            trial_ids=ids, noise_sd=0.0)
    for k in range(4):
        one = orc.transfer_run(w["layers"], w["projections"], w["cond_inputs"][k:k + 1], 1,
                               seed=2, trial_ids=np.array([3 * k], np.uint32), noise_sd=0.0)
        assert full["step"][3 * k] == one["step"][0]
        assert np.array_equal(full["y"][3 * k], one["y"][0])


# ------------------------------------------------------------ predator-prey ---

BIG = 1e12   # observation offset that makes the perception noise ~1e-12


@pytest.mark.parametrize("pos,dist", [
    # predator behind the player, opposite the prey: move straight at the prey
    ([0, 0, -3, 0, 5, 0], 4.0),
    # predator between player and prey, same line: u_prey - 0.5 u_pred points at the prey
    ([0, 0, 2, 0, 5, 0], 4.0),
    # player on the prey: any unit step ends at distance 1 (step length is 1)
    ([1, 1, 4, 5, 1, 1], 1.0),
    # perpendicular predator: act = (-1, 2)/sqrt(5)
    ([0, 0, 3, 0, 0, 4], math.sqrt(0.2 + (2 / math.sqrt(5) - 4) ** 2)),
])
def test_pp_geometry(orc, pos, dist):
    a = np.array([0.3, 0.6, 0.1])
    v, per = orc.pp_outcome(np.array(pos, np.float32), a, seed=1, trial=0, cand=0, obs_offset=BIG)
    assert math.isclose(v, -dist - float((a * a).sum()), rel_tol=1e-9, abs_tol=1e-9)
    assert np.allclose(per, pos, atol=1e-9)


def test_pp_perception_sd(orc):
    a = np.array([0.0, 0.4, 1.0])
    n = 20000
    pos = np.array([1, 2, 3, 4, 5, 6], np.float32)
    per = np.array([orc.pp_outcome(pos, a, 7, j, 11)[1] for j in range(n)])
    err = per - pos.astype(np.float64)
    for e in range(3):
        sd = 1.0 / (0.1 + a[e])
        for c in range(2):
            assert abs(err[:, 2 * e + c].var() / sd**2 - 1) < 5 * math.sqrt(2.0 / n)


def test_pp_index_layout_and_cost_order(orc):
    """No perception noise: candidates differ only by the cost sum a^2, with
    c = (l0 * L1 + l1) * L2 + l2."""
    lv = [np.array([0.0, 0.5], np.float32), np.array([0.0, 0.2, 0.9], np.float32),
          np.array([0.0, 0.1, 0.3, 0.7], np.float32)]
    pos = W.predator_prey(n_trials=8)["pos"]
    m = orc.pp_means(pos, lv, seed=4, obs_offset=BIG)
    assert m.shape == (24,)
    for c in range(24):
        l0, l1, l2 = c // 12, (c // 4) % 3, c % 4
        cost = float(lv[0][l0]) ** 2 + float(lv[1][l1]) ** 2 + float(lv[2][l2]) ** 2
        assert math.isclose(m[c] - m[0], -cost, abs_tol=1e-9)
    assert orc.argmax(m)[0] == 0


def test_pp_mean_is_trial_average(orc):
    w = W.predator_prey(n_trials=16, levels=3)
    m = orc.pp_means(w["pos"], w["levels"], seed=w["seed"])
    for c in [0, 13, 26]:
        a = np.array([w["levels"][0][c // 9], w["levels"][1][(c // 3) % 3], w["levels"][2][c % 3]],
                     np.float64)
        vals = [orc.pp_outcome(w["pos"][j], a, w["seed"], j, c)[0] for j in range(16)]
        assert math.isclose(m[c], math.fsum(vals) / 16, rel_tol=1e-14)


def test_argmax_ties_lowest_index(orc):
    v = np.array([1.0, 3.0, 2.0, 3.0, -1.0])
    b, bv, g = orc.argmax(v)
    assert b == int(np.argmax(v)) == 1 and bv == 3.0 and g == 0.0
    b, bv, g = orc.argmax(np.array([0.5, -2.0, 0.25]))
    assert b == 0 and g == 0.25
    assert orc.argmax(np.array([7.0])) == (0, 7.0, 0.0)
