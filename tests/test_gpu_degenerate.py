"""Degenerate cases on the GPU, checked against closed forms and exact
invariants rather than only against the oracle: noise-free runs (sigma = 0)
of every run kind, and a grid search at the largest level count per signal."""
import numpy as np
import pytest

from gpu_util import FLOAT_RTOL, compare_decisions, dev, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2110_15425_gb300 import binding as B
    torch.cuda.init()
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


def _run(model, n, seed, trial_params=None, cond=None, cond_block=1, state=0, mode=0):
    import torch
    from paper_2110_15425_gb300 import binding as B
    choice = torch.zeros(max(n, 1), dtype=torch.int8, device="cuda")
    step = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    fs = torch.zeros(max(n, 1) * max(state, 1), dtype=torch.float32, device="cuda")
    B.dg_run(model, B.run_desc(n, seed, trial_params=trial_params, cond_inputs=cond,
                               n_cond=0 if cond is None else cond.shape[0], cond_block=cond_block,
                               mode=mode), choice, step, fs if state else None)
    return host(choice)[:n], host(step)[:n], host(fs)[:n * state].reshape(n, state) if state else None


@pytest.mark.parametrize("mode", [0, 1])
def test_ddm_noise_free_crossing_step(ctx, orc, mode):
    """sigma = 0: x_k = k A dt, so the trial ends at the first k with
    k A dt >= z, choice 1, for every (A, z) (z / (A dt) < 10,000 here). The
    state's fixed-point block sums carry a systematic rounding of at most
    2^-29 per 4-step block, so trials whose z / (A dt) lies within 0.05 of an
    integer are left to the oracle comparison."""
    from paper_2110_15425_gb300 import binding as B
    rng = np.random.default_rng(17)
    n, dt = 5000, 1e-3
    A = rng.uniform(0.3, 1.0, n).astype(np.float32)
    z = rng.uniform(0.5, 2.0, n).astype(np.float32)
    m = B.compose_ddm(ctx, dt=dt, sigma=0.0, max_steps=10000)
    try:
        c, s, x = _run(m, n, 5, trial_params=dev(np.concatenate([A, z])), state=1, mode=mode)
    finally:
        B.dg_model_free(m)
    ratio = z.astype(np.float64) / (A.astype(np.float64) * dt)
    k = np.ceil(ratio).astype(np.int64)
    clear = np.abs(ratio - np.round(ratio)) > 0.05
    assert clear.mean() > 0.85
    assert np.all(c == 1)
    assert np.array_equal(s[clear], k[clear]), np.nonzero(s[clear] != k[clear])[0][:5]
    np.testing.assert_allclose(x[:, 0], s * A.astype(np.float64) * dt, rtol=1e-4)
    compare_decisions(c, s, orc.ddm_run(A, z, 5, dt=dt, sigma=0.0), "ddm sigma 0")


def test_ddm_noise_free_timeout(ctx):
    """sigma = 0 and z / (A dt) beyond the cap: every trial times out (choice
    -1, step = max_steps) with x = max_steps A dt (to the fixed-point block
    rounding, here 4e-5 relative)."""
    from paper_2110_15425_gb300 import binding as B
    n = 777
    A = np.full(n, 0.01, np.float32)
    z = np.full(n, 2.0, np.float32)
    m = B.compose_ddm(ctx, dt=1e-3, sigma=0.0, max_steps=10000)
    try:
        for mode in (0, 1):
            c, s, x = _run(m, n, 1, trial_params=dev(np.concatenate([A, z])), state=1, mode=mode)
            assert np.all(c == -1) and np.all(s == 10000)
            np.testing.assert_allclose(x[:, 0], 10000 * 0.01 * 1e-3, rtol=1e-4)
    finally:
        B.dg_model_free(m)


@pytest.mark.parametrize("N", [4, 16])
def test_lca_noise_free_fixed_point(ctx, N):
    """sigma = 0 with leak k above inhibition beta (test-only parameters) and
    small inputs: the state settles at x*_i = (I_i - beta S) / (k - beta),
    S = sum I / (k - beta + N beta), below the threshold, so every trial runs
    to the cap and ends there."""
    from paper_2110_15425_gb300 import binding as B
    rng = np.random.default_rng(N)
    n, k, beta = 600, 0.5, 0.02
    I = rng.uniform(0.2, 0.3, (n, N)).astype(np.float32)
    m = B.compose_lca(ctx, N, leak=k, inhibition=beta, sigma=0.0, dt=0.01, threshold=1.0,
                      max_steps=3000)
    try:
        for mode in (0, 1):
            c, s, x = _run(m, n, 3, trial_params=dev(I), state=N, mode=mode)
            Id = I.astype(np.float64)
            S = Id.sum(1, keepdims=True) / (k - beta + N * beta)
            xs = (Id - beta * S) / (k - beta)
            assert np.all(xs > 0) and np.all(xs < 1.0)
            assert np.all(c == -1) and np.all(s == 3000)
            # 3,000 steps of dt 0.01 = 30 time constants of the slowest mode
            assert rel_err(x, xs, 1.0) < 1e-4
    finally:
        B.dg_model_free(m)


def _identical_within_conditions(c, s, y, cond_of):
    for k in np.unique(cond_of):
        idx = np.nonzero(cond_of == k)[0]
        assert np.all(c[idx] == c[idx[0]]) and np.all(s[idx] == s[idx[0]]), k
        assert np.array_equal(y[idx], np.broadcast_to(y[idx[0]], y[idx].shape)), k


def test_stroop_noise_free(ctx, orc):
    """noise_sd = 0: the network is deterministic, so every trial of a
    condition ends bit-identically; the oracle agrees per trial."""
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_small(weight_seed=4, trials_per_condition=100, weight_range=6.0)
    m = B.compose_network(ctx, w["layers"], w["projections"], rate=w["rate"], noise_sd=0.0,
                          stop_layer=w["stop_layer"], stop_threshold=w["stop_threshold"],
                          max_steps=w["max_steps"])
    try:
        ss = B.dg_model_info(m)[1]
        for mode in (0, 1):
            c, s, y = _run(m, 400, w["seed"], cond=dev(w["cond_inputs"]),
                           cond_block=w["cond_block"], state=ss, mode=mode)
            _identical_within_conditions(c, s, y, np.arange(400) // 100)
            ref = orc.transfer_run(w["layers"], w["projections"], w["cond_inputs"],
                                   w["cond_block"], w["seed"], rate=w["rate"], noise_sd=0.0,
                                   stop_layer=w["stop_layer"],
                                   stop_threshold=w["stop_threshold"],
                                   max_steps=w["max_steps"], n_trials=400)
            compare_decisions(c, s, ref, "stroop noise 0")
            assert rel_err(y, ref["y"], 1e-2) < FLOAT_RTOL
    finally:
        B.dg_model_free(m)


def test_wide_noise_free(ctx):
    """noise_sd = 0 on the tensor-core wide network: trials of the same
    condition (t mod 256) end bit-identically, whatever row of whichever
    block runs them."""
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    n = 1024 + 37
    w = W.stroop_wide(n_trials=n, max_steps=120)
    m = B.compose_network(ctx, w["layers"], w["projections"], rate=w["rate"], noise_sd=0.0,
                          stop_layer=w["stop_layer"], stop_threshold=w["stop_threshold"],
                          max_steps=w["max_steps"], bf16_edges=(2,))
    try:
        c, s, y = _run(m, n, w["seed"], cond=dev(w["cond_inputs"]), cond_block=1, state=16)
        _identical_within_conditions(c, s, y, np.arange(n) % 256)
        assert (s < 120).any() and (s == 120).any()
    finally:
        B.dg_model_free(m)


def test_grid_largest_level_count(ctx, orc):
    """4,096 levels on one signal (the largest the boundary accepts) by 2 by 1:
    8,192 candidates, argmax and means against the oracle."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    g = W.predator_prey(n_trials=4, levels=2)
    lv = [np.linspace(0.0, 1.0, 4096).astype(np.float32), np.array([0.2, 0.7], np.float32),
          np.array([0.5], np.float32)]
    m = B.compose_predator_prey(ctx)
    try:
        for mode in (0, 1):
            res = torch.zeros(3, dtype=torch.float64, device="cuda")
            means = torch.zeros(8192, dtype=torch.float64, device="cuda")
            B.dg_grid_search(m, B.grid_desc([dev(x) for x in lv], dev(g["pos"]), g["seed"],
                                            mode=mode), res, means)
            ref = orc.pp_means(g["pos"], lv, g["seed"])
            got = host(means)
            assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-5
            r = host(res)
            best = int(r[:1].view(np.int64)[0])
            srt = np.sort(ref)
            if srt[-1] - srt[-2] >= 1e-5:
                assert best == int(np.argmax(ref))
            assert best == int(np.argmax(got))
    finally:
        B.dg_model_free(m)
