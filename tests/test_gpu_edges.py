"""Edge cases of every run kind against the oracle: a single trial, a step cap
of one, empty runs, trial ids at the top of the 32-bit counter range, and a
one-candidate grid."""
import numpy as np
import pytest

from gpu_util import compare_decisions, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2110_15425_gb300 import binding as B
    torch.cuda.init()
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


def _run(model, n, seed, trial_params=None, cond=None, cond_block=1, mode=0, offset=0):
    import torch
    from paper_2110_15425_gb300 import binding as B
    choice = torch.zeros(max(n, 1), dtype=torch.int8, device="cuda")
    step = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    B.dg_run(model, B.run_desc(n, seed, trial_params=trial_params, cond_inputs=cond,
                               n_cond=0 if cond is None else cond.shape[0], cond_block=cond_block,
                               mode=mode, trial_offset=offset), choice, step)
    return host(choice)[:n], host(step)[:n]


@pytest.mark.parametrize("mode", [0, 1])
def test_ddm_top_of_counter_range(ctx, orc, mode):
    """The last 5,000 trials of a 2^32-trial job: their ids fill the top of the
    Philox counter's trial word."""
    from paper_2110_15425_gb300 import binding as B
    rng = np.random.default_rng(5)
    n = 5000
    A = rng.uniform(0.1, 1.0, n).astype(np.float32)
    z = rng.uniform(0.5, 2.0, n).astype(np.float32)
    off = (1 << 32) - n
    model = B.compose_ddm(ctx)
    try:
        c, s = _run(model, n, 9, trial_params=dev(np.concatenate([A, z])), mode=mode, offset=off)
    finally:
        B.dg_model_free(model)
    ref = orc.ddm_run_offset(A, z, 9, off)
    compare_decisions(c, s, ref, "ddm top ids")


@pytest.mark.parametrize("mode", [0, 1])
def test_single_trial_every_kind(ctx, orc, mode):
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    # DDM
    w = W.ddm(n_trials=1, param_seed=4)
    m = B.compose_ddm(ctx)
    c, s = _run(m, 1, w["seed"], trial_params=dev(np.concatenate([w["A"], w["z"]])), mode=mode)
    B.dg_model_free(m)
    compare_decisions(c, s, orc.ddm_run(w["A"], w["z"], w["seed"]), "ddm 1")
    # LCA N = 4 and 16
    for N in (4, 16):
        w = W.lca(n_trials=1, N=N)
        m = B.compose_lca(ctx, N)
        c, s = _run(m, 1, w["seed"], trial_params=dev(w["I"]), mode=mode)
        B.dg_model_free(m)
        compare_decisions(c, s, orc.lca_run(w["I"], w["seed"]), f"lca{N} 1")
    # Stroop network and wide network
    for kind in ("stroop", "wide"):
        if kind == "wide" and mode == 1:
            continue
        if kind == "stroop":
            w = W.stroop_small(weight_seed=4, trials_per_condition=1, weight_range=6.0)
            proj, bf = w["projections"], ()
        else:
            import torch
            w = W.stroop_wide(n_trials=1, max_steps=60)
            s_, r_, Wr = w["projections"][2]
            proj = [w["projections"][0], w["projections"][1],
                    (s_, r_, torch.from_numpy(Wr).to(torch.bfloat16).float().numpy())]
            bf = (2,)
        m = B.compose_network(ctx, w["layers"], w["projections"], rate=w["rate"],
                              noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                              stop_threshold=w["stop_threshold"], max_steps=w["max_steps"],
                              bf16_edges=bf)
        c, s = _run(m, 1, w["seed"], cond=dev(w["cond_inputs"]), cond_block=w["cond_block"],
                    mode=mode)
        B.dg_model_free(m)
        ref = orc.transfer_run(w["layers"], proj, w["cond_inputs"], w["cond_block"], w["seed"],
                               rate=w["rate"], noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                               stop_threshold=w["stop_threshold"], max_steps=w["max_steps"],
                               n_trials=1)
        compare_decisions(c, s, ref, f"{kind} 1")


@pytest.mark.parametrize("mode", [0, 1])
def test_step_cap_of_one(ctx, orc, mode):
    """max_steps = 1: every trial ends after its first step (a decision there,
    or the timeout code)."""
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.lca(n_trials=777, N=8)
    m = B.compose_lca(ctx, 8, max_steps=1)
    c, s = _run(m, 777, w["seed"], trial_params=dev(w["I"]), mode=mode)
    B.dg_model_free(m)
    ref = orc.lca_run(w["I"], w["seed"], max_steps=1)
    compare_decisions(c, s, ref, "lca cap 1")
    assert np.all(s == 1)
    w = W.stroop_small(weight_seed=4, trials_per_condition=50, weight_range=6.0, max_steps=1)
    m = B.compose_network(ctx, w["layers"], w["projections"], rate=w["rate"],
                          noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                          stop_threshold=w["stop_threshold"], max_steps=1)
    c, s = _run(m, 200, w["seed"], cond=dev(w["cond_inputs"]), cond_block=w["cond_block"],
                mode=mode)
    B.dg_model_free(m)
    ref = orc.transfer_run(w["layers"], w["projections"], w["cond_inputs"], w["cond_block"],
                           w["seed"], rate=w["rate"], noise_sd=w["noise_sd"],
                           stop_layer=w["stop_layer"], stop_threshold=w["stop_threshold"],
                           max_steps=1, n_trials=200)
    compare_decisions(c, s, ref, "stroop cap 1")
    assert np.all(s == 1)


def test_empty_runs(ctx):
    """n_trials = 0 is a valid call for every kind and writes nothing."""
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_small()
    models = [B.compose_ddm(ctx), B.compose_lca(ctx, 4),
              B.compose_network(ctx, w["layers"], w["projections"], rate=w["rate"],
                                noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                                stop_threshold=w["stop_threshold"], max_steps=w["max_steps"])]
    try:
        for m in models:
            for mode in (0, 1):
                c, s = _run(m, 0, 1, mode=mode)
                assert c.size == 0 and s.size == 0
    finally:
        for m in models:
            B.dg_model_free(m)


def test_one_candidate_grid(ctx, orc):
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    g = W.predator_prey(n_trials=1, levels=2)
    lv = [np.array([0.3], np.float32)] * 3
    m = B.compose_predator_prey(ctx)
    try:
        for mode in (0, 1):
            res = torch.zeros(3, dtype=torch.float64, device="cuda")
            means = torch.zeros(1, dtype=torch.float64, device="cuda")
            B.dg_grid_search(m, B.grid_desc([dev(l) for l in lv], dev(g["pos"]), g["seed"],
                                            mode=mode), res, means)
            r = host(res)
            assert int(r[:1].view(np.int64)[0]) == 0 and r[2] == 0.0
            ref = orc.pp_means(g["pos"], lv, g["seed"])
            assert abs(host(means)[0] - ref[0]) <= 1e-5 * max(1.0, abs(ref[0]))
    finally:
        B.dg_model_free(m)
