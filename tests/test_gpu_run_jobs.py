"""GPU: several DDM or LCA jobs in one persistent launch (dg_run_jobs, and the
serving loop's groups of small jobs) return exactly what each job returns
when run alone, and what the oracle returns."""
import numpy as np
import pytest

from gpu_util import compare_decisions, dev, host

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 37, 1000, 4097, 20000, 3, 65536]


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2110_15425_gb300 import binding as B
    torch.cuda.init()
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


def _inputs(kind, n, i, N=None):
    from paper_2110_15425_gb300 import workloads as W
    if kind == "ddm":
        w = W.ddm(n_trials=max(n, 1), param_seed=70 + i)
        return np.ascontiguousarray(np.concatenate([w["A"][:n], w["z"][:n]]).astype(np.float32))
    w = W.lca(n_trials=max(n, 1), N=N, input_seed=90 + i)
    return np.ascontiguousarray(w["I"][:n].astype(np.float32))


def _alone(B, model, h, n, seed, offset, state):
    import torch
    d = B.run_desc(n, seed, trial_params=dev(h) if n else None, trial_offset=offset)
    c = torch.full((max(n, 1),), 9, dtype=torch.int8, device="cuda")
    s = torch.full((max(n, 1),), -9, dtype=torch.int32, device="cuda")
    f = torch.zeros(max(n, 1) * state, dtype=torch.float32, device="cuda")
    if n:
        B.dg_run(model, d, c, s, f)
    return host(c)[:n], host(s)[:n], host(f)[:n * state]


def _jobs(B, model, hs, ns, seeds, offsets, state, with_state):
    import torch
    descs, cs, ss, fs = [], [], [], []
    for h, n, seed, off, ws in zip(hs, ns, seeds, offsets, with_state):
        descs.append(B.run_desc(n, seed, trial_params=dev(h) if n else None, trial_offset=off))
        cs.append(torch.full((max(n, 1),), 9, dtype=torch.int8, device="cuda"))
        ss.append(torch.full((max(n, 1),), -9, dtype=torch.int32, device="cuda"))
        fs.append(torch.zeros(max(n, 1) * state, dtype=torch.float32, device="cuda") if ws
                  else None)
    B.dg_run_jobs(model, descs, cs, ss, fs)
    return descs, cs, ss, fs


@pytest.mark.parametrize("kind,N", [("ddm", 1), ("lca", 4), ("lca", 8), ("lca", 16), ("lca", 5),
                                    ("lca", 1)])
def test_run_jobs_equal_single_runs(ctx, kind, N):
    from paper_2110_15425_gb300 import binding as B
    if kind == "ddm":
        model = B.compose_ddm(ctx)
    elif N == 1:
        model = B.compose_lca(ctx, 1, leak=0.0, inhibition=0.0, sigma=1.0, dt=1e-3,
                              threshold=1.25, max_steps=10000, rectify=False, two_sided=True)
    else:
        model = B.compose_lca(ctx, N)
    try:
        state = B.dg_model_info(model)[1]
        hs = [_inputs(kind, n, i, N) for i, n in enumerate(SIZES)]
        seeds = [11 + 1000003 * i for i in range(len(SIZES))]
        offsets = [0, 5, 0, 123456, 0, 7, 2 ** 31, 0]
        with_state = [i % 2 == 0 for i in range(len(SIZES))]
        descs, cs, ss, fs = _jobs(B, model, hs, SIZES, seeds, offsets, state, with_state)
        for i, n in enumerate(SIZES):
            c, s, f = _alone(B, model, hs[i], n, seeds[i], offsets[i], state)
            assert np.array_equal(host(cs[i])[:n], c), (kind, N, i)
            assert np.array_equal(host(ss[i])[:n], s), (kind, N, i)
            if with_state[i]:
                assert np.array_equal(host(fs[i])[:n * state].view(np.uint32), f.view(np.uint32))
            if n == 0:
                assert host(cs[i])[0] == 9 and host(ss[i])[0] == -9   # untouched
    finally:
        B.dg_model_free(model)


def _stroop(B, ctx, weight_seed=4):
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_small(weight_seed=weight_seed)
    m = B.compose_network(ctx, w["layers"], w["projections"], rate=w["rate"],
                          noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                          stop_threshold=w["stop_threshold"], max_steps=w["max_steps"])
    return w, m


def _net_desc(B, n, seed, cond, cond_block, offset):
    return B.run_desc(n, seed, cond_inputs=dev(cond), n_cond=cond.shape[0], cond_block=cond_block,
                      trial_offset=offset)


def test_run_jobs_network_equal_single_runs(ctx):
    """Jobs of one small network, each with its own condition table, condition
    block, seed and trial offset, in one launch: each equals its dg_run."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    w, model = _stroop(B, ctx)
    try:
        state = B.dg_model_info(model)[1]
        rng = np.random.default_rng(5)
        sizes = [0, 1, 37, 1000, 4097, 20000, 3]
        jobs = []
        for i, n in enumerate(sizes):
            nc = int(rng.integers(1, 6))
            cond = rng.uniform(0, 1, (nc, w["cond_inputs"].shape[1])).astype(np.float32)
            jobs.append((n, 77 + 1000003 * i, cond, int(rng.integers(1, 300)),
                         [0, 9, 123456, 0, 5, 2 ** 30, 7][i], i % 2 == 0))
        descs = [_net_desc(B, n, sd, c, cb, off) for n, sd, c, cb, off, _ in jobs]
        cs = [torch.full((max(n, 1),), 9, dtype=torch.int8, device="cuda") for n, *_ in jobs]
        ss = [torch.full((max(n, 1),), -9, dtype=torch.int32, device="cuda") for n, *_ in jobs]
        fs = [torch.zeros(max(n, 1) * state, dtype=torch.float32, device="cuda") if ws else None
              for n, *_, ws in jobs]
        B.dg_run_jobs(model, descs, cs, ss, fs)
        for i, (n, sd, c, cb, off, ws) in enumerate(jobs):
            if n == 0:
                assert host(cs[i])[0] == 9 and host(ss[i])[0] == -9
                continue
            c1 = torch.zeros(n, dtype=torch.int8, device="cuda")
            s1 = torch.zeros(n, dtype=torch.int32, device="cuda")
            f1 = torch.zeros(n * state, dtype=torch.float32, device="cuda")
            B.dg_run(model, _net_desc(B, n, sd, c, cb, off), c1, s1, f1)
            assert np.array_equal(host(cs[i])[:n], host(c1)), i
            assert np.array_equal(host(ss[i])[:n], host(s1)), i
            if ws:
                assert np.array_equal(host(fs[i])[:n * state].view(np.uint32),
                                      host(f1).view(np.uint32)), i
    finally:
        B.dg_model_free(model)


def test_run_jobs_against_oracle(ctx, orc, threads):
    """Job i of a multi-job launch against the oracle on a sample of its
    trials, with the job's own seed and trial offset."""
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    md = B.compose_ddm(ctx)
    ml = B.compose_lca(ctx, 8)
    try:
        for kind, model in (("ddm", md), ("lca", ml)):
            ws = [W.ddm(n_trials=6000, param_seed=5 + i) if kind == "ddm"
                  else W.lca(n_trials=6000, N=8, input_seed=5 + i) for i in range(3)]
            offsets = [0, 6000, 40000]
            seeds = [w["seed"] + i for i, w in enumerate(ws)]
            hs = [np.ascontiguousarray(np.concatenate([w["A"], w["z"]])) if kind == "ddm"
                  else np.ascontiguousarray(w["I"]) for w in ws]
            state = B.dg_model_info(model)[1]
            descs, cs, ss, fs = _jobs(B, model, hs, [6000] * 3, seeds, offsets, state,
                                      [False] * 3)
            for i, w in enumerate(ws):
                ids = np.arange(0, 6000, 13, dtype=np.uint32)
                # the oracle reads trial g's inputs at row g: pad to the offset
                off = offsets[i]
                if kind == "ddm":
                    A = np.concatenate([np.zeros(off, np.float32), w["A"]])
                    z = np.concatenate([np.ones(off, np.float32), w["z"]])
                    ref = orc.ddm_run(A, z, seeds[i], trial_ids=ids + off, threads=threads)
                else:
                    I = np.concatenate([np.zeros((off, 8), np.float32), w["I"]])
                    ref = orc.lca_run(I, seeds[i], trial_ids=ids + off, threads=threads)
                compare_decisions(host(cs[i])[ids], host(ss[i])[ids], ref, f"{kind} job {i}")
    finally:
        B.dg_model_free(md)
        B.dg_model_free(ml)


def test_run_jobs_arguments(ctx):
    import torch
    from paper_2110_15425_gb300 import binding as B
    md = B.compose_ddm(ctx)
    mp = B.compose_predator_prey(ctx)
    h = _inputs("ddm", 10, 0)
    c = torch.zeros(10, dtype=torch.int8, device="cuda")
    s = torch.zeros(10, dtype=torch.int32, device="cuda")
    try:
        d = B.run_desc(10, 1, trial_params=dev(h))
        with pytest.raises(RuntimeError):
            B.dg_run_jobs(md, [], [], [])
        with pytest.raises(RuntimeError):
            B.dg_run_jobs(md, [d] * 257, [c] * 257, [s] * 257)
        with pytest.raises(RuntimeError):
            B.dg_run_jobs(mp, [d], [c], [s])
        dp = B.run_desc(10, 1, trial_params=dev(h), mode=B.DG_MODE_PLAIN)
        with pytest.raises(RuntimeError):
            B.dg_run_jobs(md, [d, dp], [c, c], [s, s])
        dn = B.run_desc(10, 1)   # no trial_params
        with pytest.raises(RuntimeError):
            B.dg_run_jobs(md, [dn], [c], [s])
        from paper_2110_15425_gb300 import workloads as W
        wd = W.stroop_wide(n_trials=10, max_steps=20)
        mw = B.compose_network(ctx, wd["layers"], wd["projections"], rate=wd["rate"],
                               noise_sd=wd["noise_sd"], stop_layer=3, stop_threshold=0.7,
                               max_steps=20, bf16_edges=(2,))
        try:   # the wide network has its own kernel: not a job-table model
            dw = B.run_desc(10, 1, cond_inputs=dev(wd["cond_inputs"]),
                            n_cond=wd["cond_inputs"].shape[0], cond_block=1)
            with pytest.raises(RuntimeError):
                B.dg_run_jobs(mw, [dw], [c], [s])
        finally:
            B.dg_model_free(mw)
        B.dg_run_jobs(md, [d] * 256, [c] * 256, [s] * 256)   # 256 jobs is the limit
    finally:
        B.dg_model_free(md)
        B.dg_model_free(mp)


@pytest.mark.parametrize("pinned", [False, True])
def test_served_small_jobs_grouped_equal_direct_runs(ctx, pinned):
    """Many small DDM and LCA jobs of several models submitted at once: the
    serving loop groups them into multi-job launches; every job's outputs
    (final states included) equal a direct dg_run of the job. With pinned host
    buffers the kernels read and write them in place (a job with any pageable
    buffer is staged through device copies, in the same group)."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    rng = np.random.default_rng(12)
    keep = []

    count = [0]

    def buf(a):
        # pinned: every seventh buffer stays pageable, so that groups mix jobs
        # used in place with staged ones
        count[0] += 1
        if not pinned or count[0] % 7 == 0:
            return a
        t = torch.from_numpy(a).pin_memory()
        keep.append(t)
        return t.numpy()
    w_st, m_st = _stroop(B, ctx)
    models = dict(ddm=B.compose_ddm(ctx), ddm2=B.compose_ddm(ctx, dt=2e-3, sigma=0.8),
                  lca4=B.compose_lca(ctx, 4), lca8=B.compose_lca(ctx, 8), stroop=m_st)
    try:
        jobs = []
        for i in range(200):
            k = ["ddm", "ddm2", "lca4", "lca8", "stroop"][int(rng.integers(5))]
            n = int(rng.integers(1, 12000))
            N = 1 if k.startswith("ddm") else 2 if k == "stroop" else int(k[3:])
            j = B.dg_job()
            j.model = models[k].value
            j.run.n_trials = n
            j.run.seed = int(rng.integers(1, 2 ** 40))
            j.run.trial_offset = int(rng.integers(0, 10 ** 6))
            if k == "stroop":
                nc = int(rng.integers(1, 5))
                h = buf(rng.uniform(0, 1, (nc, w_st["cond_inputs"].shape[1])).astype(np.float32))
                j.run.cond_inputs = h.ctypes.data
                j.run.n_cond = nc
                j.run.cond_block = int(rng.integers(1, 100))
            else:
                h = buf(_inputs("ddm" if N == 1 else "lca", n, 200 + i, N))
                j.run.trial_params = h.ctypes.data
            ch = buf(np.full(n, 9, np.int8))
            st = buf(np.full(n, -9, np.int32))
            fs = buf(np.zeros(n * N, np.float32)) if i % 3 == 0 else None
            j.choice = ch.ctypes.data
            j.step = st.ctypes.data
            if fs is not None:
                j.final_state = fs.ctypes.data
            jobs.append((k, n, N, h, j, ch, st, fs))
        tickets = [B.dg_submit(ctx, x[4]) for x in jobs]
        for t in tickets:
            r = B.dg_wait(ctx, t, 120000)
            assert r.status == 0
        for k, n, N, h, j, ch, st, fs in jobs:
            if k == "stroop":
                import torch
                c1 = torch.zeros(n, dtype=torch.int8, device="cuda")
                s1 = torch.zeros(n, dtype=torch.int32, device="cuda")
                f1 = torch.zeros(n * N, dtype=torch.float32, device="cuda")
                B.dg_run(models[k], _net_desc(B, n, j.run.seed, np.asarray(h), j.run.cond_block,
                                              j.run.trial_offset), c1, s1, f1)
                c, s, f = host(c1), host(s1), host(f1)
            else:
                c, s, f = _alone(B, models[k], h, n, j.run.seed, j.run.trial_offset, N)
            assert np.array_equal(ch, c) and np.array_equal(st, s), (k, n)
            if fs is not None:
                assert np.array_equal(fs.view(np.uint32), f.view(np.uint32)), (k, n)
    finally:
        for m in models.values():
            B.dg_model_free(m)


def test_served_grid_searches_grouped_equal_direct_searches(ctx):
    """Grid searches submitted together: those of one grid shape and trial
    count share a batched launch in the serving loop; each job's result and
    candidate means equal a direct dg_grid_search of it, bit for bit."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    model = B.compose_predator_prey(ctx)
    try:
        specs = [(12, 64)] * 20 + [(7, 64)] * 6 + [(12, 33)] * 3 + [(30, 64)]
        jobs = []
        for i, (L, T) in enumerate(specs):
            g = W.predator_prey(levels=L, pos_seed=40 + i, noise_seed=90 + i)
            pos = np.ascontiguousarray(g["pos"][:T])
            lvs = [np.ascontiguousarray(x) for x in g["levels"]]
            j = B.dg_job()
            j.model = model.value
            j.is_grid = 1
            j.grid.positions = pos.ctypes.data
            j.grid.n_trials = T
            j.grid.seed = g["seed"]
            for e in range(3):
                j.grid.levels[e] = lvs[e].ctypes.data
                j.grid.n_levels[e] = L
            res = np.zeros(3, np.float64)
            means = np.zeros(L ** 3, np.float64)
            j.grid_result = res.ctypes.data
            j.cand_means = means.ctypes.data
            jobs.append((L, T, g, pos, lvs, j, res, means))
        tickets = [B.dg_submit(ctx, x[5]) for x in jobs]
        for t in tickets:
            assert B.dg_wait(ctx, t, 120000).status == 0
        for L, T, g, pos, lvs, j, res, means in jobs:
            r2 = torch.zeros(3, dtype=torch.float64, device="cuda")
            m2 = torch.zeros(L ** 3, dtype=torch.float64, device="cuda")
            B.dg_grid_search(model, B.grid_desc([dev(x) for x in lvs], dev(pos), g["seed"]), r2, m2)
            assert np.array_equal(means, host(m2)), (L, T)
            assert np.array_equal(res, host(r2)), (L, T)
    finally:
        B.dg_model_free(model)


def test_tune_stats_count_tuned_keys_and_untuned_served_launches(monkeypatch):
    """A direct run tunes its size bucket (one more tuned key); a served job of
    an untuned bucket runs the default shape and is counted."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    monkeypatch.setenv("DG_SERVE_GROUP_TRIALS", "0")   # every served job its own launch
    c = B.dg_create(0)
    model = B.compose_ddm(c)
    try:
        keys0, untuned0 = B.dg_tune_stats(c)
        assert untuned0 == 0
        h = _inputs("ddm", 5000, 1)
        ch = torch.zeros(5000, dtype=torch.int8, device="cuda")
        st = torch.zeros(5000, dtype=torch.int32, device="cuda")
        B.dg_run(model, B.run_desc(5000, 3, trial_params=dev(h)), ch, st)
        keys1, untuned1 = B.dg_tune_stats(c)
        assert keys1 == keys0 + 1 and untuned1 == 0
        # a size bucket nothing tuned yet, through the serving thread
        n = 70000
        hs = _inputs("ddm", n, 2)
        j = B.dg_job()
        j.model = model.value
        j.run.n_trials = n
        j.run.seed = 4
        j.run.trial_params = hs.ctypes.data
        co, so = np.zeros(n, np.int8), np.zeros(n, np.int32)
        j.choice, j.step = co.ctypes.data, so.ctypes.data
        assert B.dg_wait(c, B.dg_submit(c, j), 120000).status == 0
        keys2, untuned2 = B.dg_tune_stats(c)
        assert keys2 == keys1 and untuned2 >= 1
    finally:
        B.dg_model_free(model)
        B.dg_destroy(c)
