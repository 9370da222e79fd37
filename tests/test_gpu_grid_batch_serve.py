"""GPU parity: predator-prey grid search and argmax against the oracle; CUDA
graph batches and the serving loop against single runs."""
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


def _grid(ctx, w, mode, offset=None):
    import torch
    from paper_2110_15425_gb300 import binding as B
    model = B.compose_predator_prey(ctx, obs_offset=w["obs_offset"] if offset is None else offset,
                                    pred_weight=w["pred_weight"])
    try:
        lv = [dev(l) for l in w["levels"]]
        pos = dev(w["pos"])
        nc = int(np.prod([l.shape[0] for l in w["levels"]]))
        means = torch.zeros(nc, dtype=torch.float64, device="cuda")
        res = torch.zeros(3, dtype=torch.float64, device="cuda")
        B.dg_grid_search(model, B.grid_desc(lv, pos, w["seed"], mode=mode), res, means)
        r = host(res)
        return host(means), int(r[:1].view(np.int64)[0]), float(r[1]), float(r[2])
    finally:
        B.dg_model_free(model)


def _check_best(means_ref, best, val, gap, margin=1e-5):
    b, bv, g = int(np.argmax(means_ref)), float(means_ref.max()), 0.0
    srt = np.sort(means_ref)
    g = srt[-1] - srt[-2] if srt.size > 1 else 0.0
    if g >= margin:
        assert best == b
    assert abs(val - bv) <= 1e-4 * max(1.0, abs(bv))
    assert abs(gap - g) <= 1e-4 * max(1.0, abs(bv))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("levels,trials", [(2, 4), (3, 64), (5, 37), (7, 100)])
def test_grid_tiny_brute_force(ctx, orc, threads, mode, levels, trials):
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey(n_trials=trials, levels=levels)
    m, best, val, gap = _grid(ctx, w, mode)
    ref = orc.pp_means(w["pos"], w["levels"], w["seed"], threads=threads)
    assert np.max(np.abs(m - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-5
    _check_best(ref, best, val, gap)
    assert best == int(np.argmax(m))


def test_grid_noise_free_cost_order(ctx, orc):
    """No perception noise: the cheapest allocation (index 0) wins."""
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey(n_trials=16, levels=4)
    m, best, val, gap = _grid(ctx, w, 0, offset=1e9)
    ref = orc.pp_means(w["pos"], w["levels"], w["seed"], obs_offset=1e9)
    assert best == 0
    np.testing.assert_allclose(m, ref, rtol=2e-6, atol=2e-6)


def test_grid_full_size(ctx, orc, threads):
    """27,000 candidates x 64 trials in the benchmark's configuration; the
    oracle evaluates every candidate (about 1.7 million trial evaluations)."""
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey()
    for mode in (0, 1):
        m, best, val, gap = _grid(ctx, w, mode)
        if mode == 0:
            ref = orc.pp_means(w["pos"], w["levels"], w["seed"], threads=threads)
        rel = np.abs(m - ref) / np.maximum(np.abs(ref), 1.0)
        assert rel.max() < 1e-5, rel.max()
        _check_best(ref, best, val, gap)


def test_grid_narrow_groups_ragged(ctx, orc, threads):
    """Grids of 16,384 candidates or more take eight lanes per candidate: a
    ragged one (17 x 31 x 37 = 19,499 candidates, 37 trials, so neither count
    fills the groups), whole and as two candidate ranges, through both entry
    points, against the oracle; the ranges give the whole call's means bit
    for bit."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    g = W.predator_prey(n_trials=37)
    rng = np.random.default_rng(19)
    lv = [np.sort(rng.uniform(0, 1, k)).astype(np.float32) for k in (17, 31, 37)]
    nc = 17 * 31 * 37
    ref = orc.pp_means(g["pos"], lv, g["seed"], threads=threads)
    model = B.compose_predator_prey(ctx)
    try:
        for search in (B.dg_grid_search, B.dg_grid_search_noalloc):
            res = torch.zeros(3, dtype=torch.float64, device="cuda")
            means = torch.zeros(nc, dtype=torch.float64, device="cuda")
            search(model, B.grid_desc([dev(x) for x in lv], dev(g["pos"]), g["seed"]), res, means)
            m = host(means)
            assert np.max(np.abs(m - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-5
            r = host(res)
            _check_best(ref, int(r[:1].view(np.int64)[0]), float(r[1]), float(r[2]))
            parts = []
            for b, c in ((0, 8000), (8000, nc - 8000)):
                pm = torch.zeros(c, dtype=torch.float64, device="cuda")
                search(model, B.grid_desc([dev(x) for x in lv], dev(g["pos"]), g["seed"],
                                          cand_begin=b, cand_count=c), res, pm)
                parts.append(host(pm))
            assert np.concatenate(parts).tobytes() == m.tobytes()
    finally:
        B.dg_model_free(model)


def test_argmax_ties_and_sizes(ctx):
    import torch
    from paper_2110_15425_gb300 import binding as B
    for n in [1, 2, 255, 256, 257, 100000, 1000003]:
        v = np.random.default_rng(n).normal(size=n)
        if n > 3:
            v[n // 3] = v[n - 2] = v.max() + 1.0   # exact tie: lowest index wins
        res = torch.zeros(3, dtype=torch.float64, device="cuda")
        B.dg_argmax_f64(ctx, dev(v), res)
        r = host(res)
        best = int(r[:1].view(np.int64)[0])
        assert best == int(np.argmax(v))
        if n > 3:
            assert r[2] == 0.0


# ------------------------------------------------------------------- batch ---

def _stroop_model(ctx, w):
    from paper_2110_15425_gb300 import binding as B
    return B.compose_network(ctx, w["layers"], w["projections"], rate=w["rate"],
                             noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                             stop_threshold=w["stop_threshold"], max_steps=w["max_steps"])


def test_batch_graph_equals_single_runs(ctx):
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    d = W.ddm(n_trials=50000, param_seed=3)
    l = W.lca(n_trials=20000, N=8)
    s = W.stroop_small(weight_seed=4)
    g = W.predator_prey(levels=6)
    md = B.compose_ddm(ctx)
    ml = B.compose_lca(ctx, 8)
    ms = _stroop_model(ctx, s)
    mp = B.compose_predator_prey(ctx)
    dp = dev(np.concatenate([d["A"], d["z"]]))
    lp = dev(l["I"])
    cond = dev(s["cond_inputs"])
    lv = [dev(x) for x in g["levels"]]
    pos = dev(g["pos"])
    outs = {}
    for tag in ("single", "batch"):
        o = dict(dc=torch.zeros(50000, dtype=torch.int8, device="cuda"),
                 ds=torch.zeros(50000, dtype=torch.int32, device="cuda"),
                 lc=torch.zeros(20000, dtype=torch.int8, device="cuda"),
                 ls=torch.zeros(20000, dtype=torch.int32, device="cuda"),
                 sc=torch.zeros(4000, dtype=torch.int8, device="cuda"),
                 ss=torch.zeros(4000, dtype=torch.int32, device="cuda"),
                 gr=torch.zeros(3, dtype=torch.float64, device="cuda"),
                 gm=torch.zeros(216, dtype=torch.float64, device="cuda"))
        rd = B.run_desc(50000, d["seed"], trial_params=dp)
        rl = B.run_desc(20000, l["seed"], trial_params=lp)
        rs = B.run_desc(4000, s["seed"], cond_inputs=cond, n_cond=4, cond_block=1000)
        gd = B.grid_desc(lv, pos, g["seed"])
        if tag == "single":
            B.dg_run(md, rd, o["dc"], o["ds"])
            B.dg_run(ml, rl, o["lc"], o["ls"])
            B.dg_run(ms, rs, o["sc"], o["ss"])
            B.dg_grid_search(mp, gd, o["gr"], o["gm"])
        else:
            b = B.dg_batch_create(ctx)
            B.dg_batch_add_run(b, md, rd, o["dc"], o["ds"])
            B.dg_batch_add_run(b, ml, rl, o["lc"], o["ls"])
            B.dg_batch_add_run(b, ms, rs, o["sc"], o["ss"])
            B.dg_batch_add_grid(b, mp, gd, o["gr"], o["gm"])
            with pytest.raises(B.DGError):   # no graph before the first launch
                B.dg_batch_kernels(b)
            for _ in range(3):   # capture, then replays
                for t in o.values():
                    t.zero_()
                B.dg_batch_launch(b)
            torch.cuda.synchronize()
            # one kernel per op at least, plus at most a three-kernel sort each
            assert 4 <= B.dg_batch_kernels(b) <= 4 * 4
            B.dg_batch_free(b)
        outs[tag] = {k: host(v) for k, v in o.items()}
    for k in outs["single"]:
        assert np.array_equal(outs["single"][k], outs["batch"][k]), k
    for m in (md, ml, ms, mp):
        B.dg_model_free(m)


# ----------------------------------------------------------------- serving ---

def _serve_ddm_job(B, model, A, z, seed):
    import ctypes as C
    n = A.shape[0]
    params = np.ascontiguousarray(np.concatenate([A, z]).astype(np.float32))
    out = dict(params=params, choice=np.zeros(n, np.int8), step=np.zeros(n, np.int32))
    j = B.dg_job()
    j.model = model.value
    j.is_grid = 0
    j.run.n_trials = n
    j.run.seed = seed
    j.run.trial_params = params.ctypes.data
    j.run.mode = 0
    j.choice = out["choice"].ctypes.data
    j.step = out["step"].ctypes.data
    return j, out


def test_serving_results_equal_alone_and_in_mix(ctx):
    """Continuous batching: each job's result is identical whether it runs
    alone or with others overlapping on the device."""
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    model = B.compose_ddm(ctx)
    sizes = [1000, 70000, 3000, 250000, 17, 40000]
    ws = [W.ddm(n_trials=n, param_seed=10 + i) for i, n in enumerate(sizes)]
    alone = []
    for w in ws:
        j, o = _serve_ddm_job(B, model, w["A"], w["z"], w["seed"])
        t = B.dg_submit(ctx, j)
        B.dg_wait(ctx, t)
        alone.append(o)
    mix, tickets = [], []
    for w in ws:
        j, o = _serve_ddm_job(B, model, w["A"], w["z"], w["seed"])
        tickets.append(B.dg_submit(ctx, j))
        mix.append(o)
    for t in tickets:
        r = B.dg_wait(ctx, t, 60000)
        assert r.status == 0 and r.t_done >= r.t_admit >= r.t_submit
    for a, b in zip(alone, mix):
        assert np.array_equal(a["choice"], b["choice"])
        assert np.array_equal(a["step"], b["step"])
    B.dg_model_free(model)


def test_serving_budget_admission(ctx):
    """A budget that fits one job at a time: jobs queue, run one by one, and
    all complete; a job larger than the budget is refused."""
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    small = B.dg_create(0, 4 * 1024 * 1024)   # 4 MB budget
    try:
        model = B.compose_ddm(small)
        jobs, tickets = [], []
        for i in range(5):
            w = W.ddm(n_trials=200000, param_seed=20 + i)   # ~2.6 MB each
            j, o = _serve_ddm_job(B, model, w["A"], w["z"], w["seed"])
            jobs.append((j, o))
            tickets.append(B.dg_submit(small, j))
        results = [B.dg_wait(small, t, 120000) for t in tickets]
        for a, b in zip(results, results[1:]):
            assert b.t_admit >= a.t_done - 1e-3   # one at a time under this budget
        w = W.ddm(n_trials=1000000)
        j, o = _serve_ddm_job(B, model, w["A"], w["z"], w["seed"])
        with pytest.raises(B.DGError) as e:
            B.dg_submit(small, j)
        assert e.value.status == B.DG_E_BUDGET
        B.dg_model_free(model)
    finally:
        B.dg_destroy(small)


def test_wait_timeout_status(ctx):
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    model = B.compose_ddm(ctx, max_steps=10000)
    w = W.ddm(n_trials=1 << 20)
    j, o = _serve_ddm_job(B, model, w["A"], w["z"], w["seed"])
    t = B.dg_submit(ctx, j)
    with pytest.raises(B.DGError) as e:
        B.dg_wait(ctx, t, 0)
    assert e.value.status == B.DG_E_TIMEOUT
    B.dg_wait(ctx, t, 120000)
    B.dg_model_free(model)


def test_trial_order_is_a_permutation_for_many_inputs(ctx):
    """The longest-expected-first order must hand out every trial exactly
    once for any inputs: batched (ordered) and plain (unordered) runs agree bit
    for bit on many input sets and sizes, including keys on bucket edges."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    ml = B.compose_lca(ctx, 8)
    md = B.compose_ddm(ctx)
    for i, n in enumerate([4096, 4097, 42018, 45761, 70001]):
        l = W.lca(n_trials=n, N=8, input_seed=1000 + i)
        d = W.ddm(n_trials=n, param_seed=2000 + i)
        for model, params in ((ml, dev(l["I"])), (md, dev(np.concatenate([d["A"], d["z"]])))):
            outs = []
            for mode in (0, 1):
                ch = torch.full((n,), 99, dtype=torch.int8, device="cuda")
                st = torch.full((n,), -7, dtype=torch.int32, device="cuda")
                B.dg_run(model, B.run_desc(n, 5 + i, trial_params=params, mode=mode), ch, st)
                outs.append((host(ch), host(st)))
            assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
            assert outs[0][1].min() >= 1
    B.dg_model_free(ml)
    B.dg_model_free(md)


def test_served_mix_of_every_kind_equals_direct_runs(ctx):
    """Jobs of every model kind submitted together (overlapping on the
    device) return exactly what a direct dg_run / dg_grid_search returns."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    s = W.stroop_small(weight_seed=4)
    wd = W.stroop_wide(n_trials=3000, max_steps=150)
    models = dict(
        ddm=B.compose_ddm(ctx), lca=B.compose_lca(ctx, 8), pp=B.compose_predator_prey(ctx),
        stroop=B.compose_network(ctx, s["layers"], s["projections"], rate=s["rate"],
                                 noise_sd=s["noise_sd"], stop_layer=5, stop_threshold=0.7,
                                 max_steps=500),
        wide=B.compose_network(ctx, wd["layers"], wd["projections"], rate=wd["rate"],
                               noise_sd=wd["noise_sd"], stop_layer=3, stop_threshold=0.7,
                               max_steps=150, bf16_edges=(2,)))
    specs = []
    for i, n in enumerate([20000, 45761, 3000, 60000, 8000, 1500]):
        specs.append(("ddm", n, W.ddm(n_trials=n, param_seed=40 + i)))
        specs.append(("lca", n, W.lca(n_trials=n, N=8, input_seed=60 + i)))
    specs.append(("stroop", 4000, s))
    specs.append(("wide", 3000, wd))
    jobs = []
    for k, n, w in specs:
        j = B.dg_job()
        j.model = models[k].value
        if k == "ddm":
            h = np.ascontiguousarray(np.concatenate([w["A"], w["z"]]))
            j.run.trial_params = h.ctypes.data
        elif k == "lca":
            h = np.ascontiguousarray(w["I"])
            j.run.trial_params = h.ctypes.data
        else:
            h = np.ascontiguousarray(w["cond_inputs"])
            j.run.cond_inputs = h.ctypes.data
            j.run.n_cond = h.shape[0]
            j.run.cond_block = w["cond_block"]
        j.run.n_trials = n
        j.run.seed = 3
        ch = np.zeros(n, np.int8)
        st = np.full(n, -7, np.int32)
        j.choice = ch.ctypes.data
        j.step = st.ctypes.data
        jobs.append((k, n, w, j, h, ch, st))
    g = W.predator_prey(levels=12)
    gj = B.dg_job()
    gj.model = models["pp"].value
    gj.is_grid = 1
    pos = np.ascontiguousarray(g["pos"])
    lvs = [np.ascontiguousarray(x) for x in g["levels"]]
    gj.grid.positions = pos.ctypes.data
    gj.grid.n_trials = 64
    gj.grid.seed = g["seed"]
    for i in range(3):
        gj.grid.levels[i] = lvs[i].ctypes.data
        gj.grid.n_levels[i] = 12
    gres = np.zeros(3, np.float64)
    gmeans = np.zeros(12 ** 3, np.float64)
    gj.grid_result = gres.ctypes.data
    gj.cand_means = gmeans.ctypes.data
    tickets = [B.dg_submit(ctx, j[3]) for j in jobs] + [B.dg_submit(ctx, gj)]
    for t in tickets:
        B.dg_wait(ctx, t, 120000)
    for k, n, w, j, h, ch, st in jobs:
        d = B.run_desc(n, 3, trial_params=dev(h) if k in ("ddm", "lca") else None,
                       cond_inputs=dev(h) if k in ("stroop", "wide") else None,
                       n_cond=h.shape[0] if k in ("stroop", "wide") else 0,
                       cond_block=w.get("cond_block", 1) if k in ("stroop", "wide") else 1)
        c2 = torch.zeros(n, dtype=torch.int8, device="cuda")
        s2 = torch.zeros(n, dtype=torch.int32, device="cuda")
        B.dg_run(models[k], d, c2, s2)
        assert np.array_equal(ch, host(c2)), (k, n)
        assert np.array_equal(st, host(s2)), (k, n)
    m2 = torch.zeros(12 ** 3, dtype=torch.float64, device="cuda")
    r2 = torch.zeros(3, dtype=torch.float64, device="cuda")
    B.dg_grid_search(models["pp"], B.grid_desc([dev(x) for x in lvs], dev(pos), g["seed"]), r2, m2)
    assert np.array_equal(gmeans, host(m2)) and np.array_equal(gres, host(r2))
    for m in models.values():
        B.dg_model_free(m)
