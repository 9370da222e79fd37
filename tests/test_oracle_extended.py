"""Pins of the oracle's Extended Stroop model (Sec. 5: two DDM nodes on the
Stroop network's response layer decide the trial)."""
import numpy as np

from paper_2110_15425_gb300 import workloads as W


def _run(orc, w, n=None, sigma=None, W_=None, bias=None, bound=None, ids=None, threads=1):
    q = (w["ddm_W"] if W_ is None else W_).shape[0]
    return orc.extended_run(
        w["layers"], w["projections"], w["cond_inputs"], w["cond_block"], w["seed"],
        w["ddm_W"] if W_ is None else W_, [w["ddm_bias"] if bias is None else bias] * q,
        [w["ddm_dt"]] * q, [w["ddm_sigma"] if sigma is None else sigma] * q,
        [w["ddm_bound"] if bound is None else bound] * q, [w["ddm_max"]] * q,
        rate=w["rate"], noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
        stop_threshold=w["stop_threshold"], max_steps=w["max_steps"], trial_ids=ids,
        n_trials=n, threads=threads)


def test_network_part_is_the_stroop_run(orc, threads):
    w = W.extended_stroop(weight_seed=4, trials_per_condition=50)
    r = _run(orc, w, n=200, threads=threads)
    s = orc.transfer_run(w["layers"], w["projections"], w["cond_inputs"], w["cond_block"],
                         w["seed"], rate=w["rate"], noise_sd=w["noise_sd"],
                         stop_layer=w["stop_layer"], stop_threshold=w["stop_threshold"],
                         max_steps=w["max_steps"], n_trials=200, threads=threads)
    assert np.array_equal(r["s_choice"], s["choice"]) and np.array_equal(r["s_step"], s["step"])
    assert np.array_equal(r["y"], s["y"])


def test_noise_free_nodes_closed_form(orc):
    """With sigma = 0 node q moves by drift_q dt per step, drift_q = bias +
    W_q . y: it reaches its bound after ceil(z / (|drift| dt)) steps on the side
    of the drift's sign, and the faster node decides the trial."""
    w = W.extended_stroop(weight_seed=4, trials_per_condition=50)
    Wd = np.array([[3.0, -3.0], [-0.5, 1.0]], np.float32)
    r = _run(orc, w, n=200, sigma=0.0, W_=Wd, bias=0.05)
    for k in range(200):
        drift = np.full(2, float(np.float32(0.05)))      # the bias is an FP32 parameter
        for i in range(2):
            drift = drift + Wd[:, i].astype(np.float64) * r["y"][k, i]
        np.testing.assert_array_equal(r["drift"][k], drift)
        steps = np.ceil(1.0 / (np.abs(drift) * 1e-3))
        for q in range(2):
            if abs(steps[q] - 1.0 / (abs(drift[q]) * 1e-3)) < 1e-6 or steps[q] > 10000:
                continue   # an exact multiple (rounding decides) or a timeout
            assert r["d_step"][k, q] == steps[q]
            assert r["d_choice"][k, q] == (1 if drift[q] > 0 else 0)
        first = int(np.argmin(r["d_step"][k]))   # argmin: lower q on equal steps
        assert r["choice"][k] == 2 * first + r["d_choice"][k, first]
        assert r["step"][k] == r["s_step"][k] + r["d_step"][k, first]


def test_nodes_draw_their_own_streams(orc):
    """Node q integrates the normals of stream (trial, cand 1 + q): a numpy
    restatement of the walk on those normals ends where the oracle's does."""
    w = W.extended_stroop(weight_seed=4, trials_per_condition=10)
    r = _run(orc, w, n=40)
    dt, z = w["ddm_dt"], w["ddm_bound"]
    for k in range(40):
        for q in range(2):
            n = int(r["d_step"][k, q])
            eps = orc.normals(w["seed"], k, 1 + q, 0, n)
            x = 0.0
            for j in range(n):
                x = x + (r["drift"][k, q] * dt + np.sqrt(dt) * eps[j])
            assert x == r["d_x"][k, q]
            if r["d_choice"][k, q] >= 0:
                assert abs(x) >= z and (r["d_choice"][k, q] == 1) == (x > 0)


def test_response_rule_and_timeout(orc):
    w = W.extended_stroop(weight_seed=4, trials_per_condition=10)
    r = _run(orc, w, n=40)
    for k in range(40):
        dec = [q for q in range(2) if r["d_choice"][k, q] >= 0]
        if dec:
            first = min(dec, key=lambda q: (r["d_step"][k, q], q))
            assert r["choice"][k] == 2 * first + r["d_choice"][k, first]
    # unreachable bounds: no node decides
    r = _run(orc, w, n=8, bound=1e6)
    assert np.all(r["choice"] == -1) and np.all(r["step"] == r["s_step"] + w["ddm_max"])


def test_equal_steps_go_to_the_lower_node(orc):
    """Node 1's drift is exactly minus node 0's: both reach a bound at the same
    step (noise-free), and the trial's response is node 0's."""
    w = W.extended_stroop(weight_seed=4, trials_per_condition=10)
    Wd = np.array([[2.0, -1.0], [-2.0, 1.0]], np.float32)
    r = _run(orc, w, n=40, sigma=0.0, W_=Wd, bias=0.0)
    both = r["d_step"][:, 0] == r["d_step"][:, 1]
    assert both.all()
    dec = r["d_choice"][:, 0] >= 0
    assert dec.any()
    assert np.all(r["choice"][dec] == r["d_choice"][dec, 0])
    assert np.all(r["d_choice"][dec, 1] == 1 - r["d_choice"][dec, 0])
