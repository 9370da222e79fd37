"""GPU: failure detection without a fault, and exact resume / sharding.

- A device wait that runs out (nothing arrives on its barrier) is reported as
  DG_E_TIMEOUT by dg_stream_status, and the context keeps working.
- A job split into several calls with trial_offset (resume at any trial, or
  a shard of a larger job) reproduces the whole job bit for bit; a grid search
  split into candidate ranges reproduces the full search.
"""
import numpy as np
import pytest

from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2110_15425_gb300 import binding as B
    torch.cuda.init()
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


def _ddm(B, torch, model, params, n, offset, seed=11):
    ch = torch.zeros(n, dtype=torch.int8, device="cuda")
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    B.dg_run(model, B.run_desc(n, seed, trial_params=params, trial_offset=offset), ch, st)
    return host(ch), host(st)


def test_device_wait_timeout_reported_and_context_survives(ctx):
    import torch
    from paper_2110_15425_gb300 import binding as B
    B.dg_stream_status(ctx)                      # clean start
    B.dg_selftest_wait_timeout(ctx, 50000)       # 50 ms wait that nothing ends
    with pytest.raises(B.DGError) as e:
        B.dg_stream_status(ctx)
    assert e.value.status == B.DG_E_TIMEOUT
    B.dg_stream_status(ctx)                      # the status word was cleared
    from paper_2110_15425_gb300 import workloads as W
    w = W.ddm(n_trials=5000)
    model = B.compose_ddm(ctx)
    c, s = _ddm(B, torch, model, dev(np.concatenate([w["A"], w["z"]])), 5000, 0)
    assert s.min() >= 1
    B.dg_stream_status(ctx)
    B.dg_model_free(model)


def test_resume_ddm_lca_stroop_at_any_trial(ctx):
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    n = 30000
    cuts = [0, 7, 12345, 20000, n]
    w = W.ddm(n_trials=n)
    md = B.compose_ddm(ctx)
    whole = _ddm(B, torch, md, dev(np.concatenate([w["A"], w["z"]])), n, 0)
    parts = [_ddm(B, torch, md, dev(np.concatenate([w["A"][a:b], w["z"][a:b]])), b - a, a)
             for a, b in zip(cuts, cuts[1:])]
    assert np.array_equal(whole[0], np.concatenate([p[0] for p in parts]))
    assert np.array_equal(whole[1], np.concatenate([p[1] for p in parts]))
    B.dg_model_free(md)

    l = W.lca(n_trials=n, N=8)
    ml = B.compose_lca(ctx, 8)

    def lca(a, b):
        ch = torch.zeros(b - a, dtype=torch.int8, device="cuda")
        st = torch.zeros(b - a, dtype=torch.int32, device="cuda")
        B.dg_run(ml, B.run_desc(b - a, 5, trial_params=dev(l["I"][a:b]), trial_offset=a), ch, st)
        return host(ch), host(st)
    whole = lca(0, n)
    parts = [lca(a, b) for a, b in zip(cuts, cuts[1:])]
    assert np.array_equal(whole[1], np.concatenate([p[1] for p in parts]))
    B.dg_model_free(ml)

    s = W.stroop_small(weight_seed=4)
    ms = B.compose_network(ctx, s["layers"], s["projections"], rate=s["rate"],
                           noise_sd=s["noise_sd"], stop_layer=5, stop_threshold=0.7, max_steps=500)
    cond = dev(s["cond_inputs"])

    def stroop(a, b):
        ch = torch.zeros(b - a, dtype=torch.int8, device="cuda")
        st = torch.zeros(b - a, dtype=torch.int32, device="cuda")
        B.dg_run(ms, B.run_desc(b - a, 1, cond_inputs=cond, n_cond=4, cond_block=1000,
                                trial_offset=a), ch, st)
        return host(ch), host(st)
    whole = stroop(0, 4000)
    parts = [stroop(a, b) for a, b in [(0, 999), (999, 1001), (1001, 4000)]]
    assert np.array_equal(whole[0], np.concatenate([p[0] for p in parts]))
    assert np.array_equal(whole[1], np.concatenate([p[1] for p in parts]))
    B.dg_model_free(ms)


def test_grid_candidate_ranges_reassemble_the_full_search(ctx):
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    from paper_2110_15425_gb300.sharding import combine_top2, shard_range
    g = W.predator_prey(levels=20)
    m = B.compose_predator_prey(ctx)
    lv = [dev(x) for x in g["levels"]]
    pos = dev(g["pos"])
    nc = 8000

    def grid(a, b):
        means = torch.zeros(b - a, dtype=torch.float64, device="cuda")
        res = torch.zeros(3, dtype=torch.float64, device="cuda")
        B.dg_grid_search(m, B.grid_desc(lv, pos, g["seed"], cand_begin=a, cand_count=b - a),
                         res, means)
        r = host(res)
        return host(means), (float(r[1]), int(r[:1].view(np.int64)[0]), float(r[1] - r[2]))
    full_m, full_r = grid(0, nc)
    spans = [shard_range(nc, k, 3) for k in range(3)]
    parts = [grid(a, b) for a, b in spans]
    assert np.array_equal(full_m, np.concatenate([p[0] for p in parts]))
    best_v, best_i, gap = combine_top2([p[1] for p in parts])
    assert best_i == full_r[1] and best_v == full_r[0]
    assert abs(gap - (full_r[0] - full_r[2])) < 1e-12
    B.dg_model_free(m)


def test_ddm_start_point_and_noise_free(ctx, orc):
    import torch
    from paper_2110_15425_gb300 import binding as B
    from gpu_util import compare_decisions
    rng = np.random.default_rng(4)
    n = 2000
    A = rng.uniform(-1, 1, n).astype(np.float32)
    z = rng.uniform(0.5, 2, n).astype(np.float32)
    for x0, sigma in [(0.3, 1.0), (-0.2, 0.5), (0.0, 0.0)]:
        model = B.compose_ddm(ctx, sigma=sigma, x0=x0, max_steps=5000)
        ch = torch.zeros(n, dtype=torch.int8, device="cuda")
        st = torch.zeros(n, dtype=torch.int32, device="cuda")
        B.dg_run(model, B.run_desc(n, 9, trial_params=dev(np.concatenate([A, z]))), ch, st)
        ref = orc.ddm_run(A, z, 9, sigma=sigma, x0=x0, max_steps=5000)
        compare_decisions(host(ch), host(st), ref, f"x0={x0} sigma={sigma}")
        B.dg_model_free(model)
