"""A batch of grid searches in one launch (dg_grid_search_batch) gives, search
by search, exactly what dg_grid_search gives: the same FP64 means bit for bit,
best index, best value and runner-up gap. Both grid forms are covered (eight
lanes per candidate from 16,384 candidates up, a warp below)."""
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


def _searches(levels, n_trials, count, seed0):
    from paper_2110_15425_gb300 import workloads as W
    out = []
    for i in range(count):
        w = W.predator_prey(n_trials=n_trials, levels=levels, pos_seed=100 + seed0 + i,
                            noise_seed=7 * i + seed0)
        # distinct level values per search: every search its own grid
        w["levels"] = [np.clip(l * (1.0 - 0.01 * i) + 0.001 * e, 0, 1).astype(np.float32)
                       for e, l in enumerate(w["levels"])]
        out.append(w)
    return out


@pytest.mark.parametrize("levels,n_trials,count", [(30, 64, 9), (9, 37, 5), (26, 1, 3), (2, 5, 2)])
def test_batch_equals_single_searches(ctx, levels, n_trials, count):
    import torch
    from paper_2110_15425_gb300 import binding as B
    model = B.compose_predator_prey(ctx)
    try:
        ws = _searches(levels, n_trials, count, levels)
        nc = levels ** 3
        keep, descs = [], []
        for w in ws:
            lv = [dev(l) for l in w["levels"]]
            pos = dev(w["pos"])
            keep.append((lv, pos))
            descs.append(B.grid_desc(lv, pos, w["seed"]))
        res = torch.zeros(count * 3, dtype=torch.float64, device="cuda")
        means = [torch.zeros(nc, dtype=torch.float64, device="cuda") for _ in ws]
        # the middle search without means
        means_arg = [m if i != count // 2 else None for i, m in enumerate(means)]
        B.dg_grid_search_batch(model, descs, res, means_arg)
        got = host(res).reshape(count, 3)
        for i, (w, d) in enumerate(zip(ws, descs)):
            r1 = torch.zeros(3, dtype=torch.float64, device="cuda")
            m1 = torch.zeros(nc, dtype=torch.float64, device="cuda")
            B.dg_grid_search(model, d, r1, m1)
            ref = host(r1)
            assert got[i, :1].view(np.int64)[0] == ref[:1].view(np.int64)[0], i
            assert got[i, 1].tobytes() == ref[1].tobytes(), i
            assert got[i, 2].tobytes() == ref[2].tobytes(), i
            if i != count // 2:
                assert np.array_equal(host(means[i]).view(np.uint64), host(m1).view(np.uint64)), i
    finally:
        B.dg_model_free(model)


def test_batch_rejects_mixed_shapes(ctx):
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    model = B.compose_predator_prey(ctx)
    try:
        a, b = W.predator_prey(levels=5), W.predator_prey(levels=6)
        keep = [([dev(l) for l in w["levels"]], dev(w["pos"])) for w in (a, b)]
        descs = [B.grid_desc(lv, pos, 1) for lv, pos in keep]
        res = torch.zeros(6, dtype=torch.float64, device="cuda")
        with pytest.raises(B.DGError) as e:
            B.dg_grid_search_batch(model, descs, res)
        assert e.value.status == B.DG_E_ARG
        d = B.grid_desc(keep[0][0], keep[0][1], 1, cand_begin=3, cand_count=5)
        with pytest.raises(B.DGError) as e:
            B.dg_grid_search_batch(model, [d], res)
        assert e.value.status == B.DG_E_ARG
    finally:
        B.dg_model_free(model)
