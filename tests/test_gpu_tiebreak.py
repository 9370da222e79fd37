"""GPU parity of the reservoir tie-break (Sec. 3.3: a random choice among
equally good parameter settings, by reservoir sampling) against the oracle's
one-pass Algorithm R."""
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


def _res(r):
    return int(r[:1].view(np.int64)[0]), float(r[1]), float(r[2])


def _planted(n, m, rng):
    """n values, the maximum repeated m times at random positions, and a
    second group of equal values below it."""
    v = np.round(rng.normal(size=n), 2)          # many exact duplicates below the top
    top = v.max() + 1.0
    v[rng.choice(n, min(m, n), replace=False)] = top
    return v


@pytest.mark.parametrize("n", [1, 2, 5, 1023, 1024, 1025, 27000, 100003])
def test_argmax_reservoir_planted_ties(ctx, orc, n):
    import torch
    from paper_2110_15425_gb300 import binding as B
    rng = np.random.default_rng(n)
    for m in (1, 2, 3, 33, 1500, n):
        if m > n:
            continue
        v = _planted(n, m, rng)
        for seed in (0, 12345, 2**37 + 11):
            res = torch.zeros(3, dtype=torch.float64, device="cuda")
            B.dg_argmax_f64_reservoir(ctx, dev(v), seed, res)
            b, bv, g = _res(host(res))
            rb, rbv, rg, k = orc.argmax_reservoir(v, seed)
            assert (b, bv, g) == (rb, rbv, rg), (n, m, seed)
            assert k == m


def test_argmax_reservoir_negative_and_all_equal(ctx, orc):
    import torch
    from paper_2110_15425_gb300 import binding as B
    for v in (np.full(5000, -3.25), np.array([-1.0, -1.0]), np.array([-np.inf, 2.0, 2.0])):
        res = torch.zeros(3, dtype=torch.float64, device="cuda")
        B.dg_argmax_f64_reservoir(ctx, dev(v), 99, res)
        assert _res(host(res)) == orc.argmax_reservoir(v, 99)[:3]


def _tie_workload(levels_zero, levels_rest, n_trials=16):
    """Perception noise scaled away (observation offset 1e30) and several
    attention levels equal to 0: every zero-cost allocation has exactly the
    same outcome on every trial, so the best mean is tied on both sides."""
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey(n_trials=n_trials, levels=2)
    lv = np.array([0.0] * levels_zero + list(levels_rest), np.float32)
    w["levels"] = [lv.copy(), lv.copy(), lv.copy()]
    w["obs_offset"] = 1e30
    return w


def _grid(ctx, w, mode, tie_break, cand_begin=0, cand_count=0, noalloc=False, with_means=True):
    import torch
    from paper_2110_15425_gb300 import binding as B
    model = B.compose_predator_prey(ctx, obs_offset=w["obs_offset"], pred_weight=w["pred_weight"])
    try:
        lv = [dev(l) for l in w["levels"]]
        nc = int(np.prod([l.shape[0] for l in w["levels"]]))
        cnt = cand_count or nc
        means = torch.zeros(cnt, dtype=torch.float64, device="cuda") if with_means else None
        res = torch.zeros(3, dtype=torch.float64, device="cuda")
        d = B.grid_desc(lv, dev(w["pos"]), w["seed"], mode=mode, cand_begin=cand_begin,
                        cand_count=cand_count, tie_break=tie_break)
        (B.dg_grid_search_noalloc if noalloc else B.dg_grid_search)(model, d, res, means)
        return (host(means) if with_means else None), _res(host(res))
    finally:
        B.dg_model_free(model)


@pytest.mark.parametrize("zeros,rest", [(2, [0.5]), (3, [0.25, 0.5, 1.0]), (10, np.arange(1, 21) / 20)])
def test_grid_reservoir_on_exact_ties(ctx, orc, threads, zeros, rest):
    w = _tie_workload(zeros, rest)
    ref = orc.pp_means(w["pos"], w["levels"], w["seed"], obs_offset=w["obs_offset"],
                       threads=threads)
    rb, rbv, rg, k = orc.argmax_reservoir(ref, w["seed"])
    assert k == zeros ** 3 and rg == 0.0
    for mode in (0, 1):
        for noalloc in (False, True):
            for with_means in (True, False):
                m, (b, bv, g) = _grid(ctx, w, mode, 1, noalloc=noalloc, with_means=with_means)
                assert b == rb and g == 0.0, (mode, noalloc, with_means, b, rb)
                if m is not None:
                    # the tie set itself is the same on both sides
                    assert np.array_equal(np.flatnonzero(m == m.max()),
                                          np.flatnonzero(ref == ref.max()))
        # lowest-index rule on the same workload
        _, (b0, _, _) = _grid(ctx, w, mode, 0)
        assert b0 == int(np.flatnonzero(ref == ref.max())[0])


def test_grid_reservoir_sub_range(ctx, orc, threads):
    """A call over candidates [b, b + c) draws with global indices: the oracle's
    pass over the full vector with -inf outside the range gives the same pick."""
    w = _tie_workload(4, [0.5, 1.0])
    ref = orc.pp_means(w["pos"], w["levels"], w["seed"], obs_offset=w["obs_offset"],
                       threads=threads)
    n = ref.shape[0]
    for b0, c in ((1, n - 1), (5, 60), (37, 100)):
        masked = np.full(n, -np.inf)
        masked[b0:b0 + c] = ref[b0:b0 + c]
        rb = orc.argmax_reservoir(masked, w["seed"])[0]
        for mode in (0, 1):
            _, (b, _, _) = _grid(ctx, w, mode, 1, cand_begin=b0, cand_count=c)
            assert b == rb, (b0, c, mode)


def test_grid_reservoir_without_ties_is_unchanged(ctx):
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey(levels=9)
    for mode in (0, 1):
        m0, r0 = _grid(ctx, w, mode, 0)
        m1, r1 = _grid(ctx, w, mode, 1)
        assert r0 == r1 and np.array_equal(m0, m1)


def test_grid_reservoir_served_and_batched(ctx, orc, threads):
    import torch
    from paper_2110_15425_gb300 import binding as B
    w = _tie_workload(5, [0.5])
    ref = orc.pp_means(w["pos"], w["levels"], w["seed"], obs_offset=w["obs_offset"],
                       threads=threads)
    rb = orc.argmax_reservoir(ref, w["seed"])[0]
    model = B.compose_predator_prey(ctx, obs_offset=w["obs_offset"], pred_weight=w["pred_weight"])
    try:
        L = w["levels"][0].shape[0]
        pos = np.ascontiguousarray(w["pos"])
        lvs = [np.ascontiguousarray(x) for x in w["levels"]]
        j = B.dg_job()
        j.model = model.value
        j.is_grid = 1
        j.grid.positions = pos.ctypes.data
        j.grid.n_trials = pos.shape[0]
        j.grid.seed = w["seed"]
        j.grid.tie_break = B.DG_TIE_RESERVOIR
        for i in range(3):
            j.grid.levels[i] = lvs[i].ctypes.data
            j.grid.n_levels[i] = L
        gres = np.zeros(3, np.float64)
        j.grid_result = gres.ctypes.data
        B.dg_wait(ctx, B.dg_submit(ctx, j), 120000)
        assert _res(gres)[0] == rb
        b = B.dg_batch_create(ctx)
        res = torch.zeros(3, dtype=torch.float64, device="cuda")
        gd = B.grid_desc([dev(x) for x in lvs], dev(pos), w["seed"], tie_break=B.DG_TIE_RESERVOIR)
        B.dg_batch_add_grid(b, model, gd, res, None)
        B.dg_batch_launch(b)
        assert _res(host(res))[0] == rb
        B.dg_batch_free(b)
    finally:
        B.dg_model_free(model)


def test_bad_tie_break_rejected(ctx):
    import torch
    from paper_2110_15425_gb300 import binding as B
    w = _tie_workload(2, [0.5])
    model = B.compose_predator_prey(ctx, obs_offset=1.0)
    try:
        res = torch.zeros(3, dtype=torch.float64, device="cuda")
        d = B.grid_desc([dev(l) for l in w["levels"]], dev(w["pos"]), 1, tie_break=7)
        with pytest.raises(B.DGError):
            B.dg_grid_search(model, d, res, None)
    finally:
        B.dg_model_free(model)
