"""The allocation-free grid search (dg_grid_search_noalloc), called through
the C ABI, gives the same results as dg_grid_search. It is meant for callers
that must not allocate device memory (open graph captures of another
framework, allocators that own the device budget, latency-bound loops), so it
works from a fixed array in the library's own device memory; two calls in a
row check that the reused array is cleared where it must be.

Both entry points run the same kernels, and a candidate's mean keeps its bits
whatever range or launch shape a call uses, so every output is compared bit
for bit: the means, the best index, its value and the runner-up gap."""
import numpy as np
import pytest

from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _run(B, fn, model, w, mode, with_means, cand_begin=0, cand_count=0):
    import torch
    lv = [dev(l) for l in w["levels"]]
    pos = dev(w["pos"])
    nc = cand_count or int(np.prod([l.shape[0] for l in w["levels"]]))
    means = torch.zeros(nc, dtype=torch.float64, device="cuda") if with_means else None
    res = torch.zeros(3, dtype=torch.float64, device="cuda")
    d = B.grid_desc(lv, pos, w["seed"], mode=mode)
    d.cand_begin, d.cand_count = cand_begin, cand_count
    fn(model, d, res, means)
    r = host(res)
    return (host(means) if with_means else None), int(r[:1].view(np.int64)[0]), r[1], r[2]


def _same(got, ref, with_means):
    if with_means:
        assert np.array_equal(got[0].view(np.uint64), ref[0].view(np.uint64))
    assert got[1] == ref[1]
    assert np.float64(got[2]).tobytes() == np.float64(ref[2]).tobytes()
    assert np.float64(got[3]).tobytes() == np.float64(ref[3]).tobytes()


@pytest.mark.parametrize("mode,with_means", [(0, True), (0, False), (1, False), (1, True)])
def test_noalloc_grid_matches_grid_search(mode, with_means):
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    torch.cuda.init()
    ctx = B.dg_create(0)
    try:
        model = B.compose_predator_prey(ctx)
        for levels, seed in [(30, 13), (11, 99)]:   # two calls in a row, different sizes
            w = W.predator_prey(levels=levels, noise_seed=seed)
            ref = _run(B, B.dg_grid_search, model, w, mode, True)
            got = _run(B, B.dg_grid_search_noalloc, model, w, mode, with_means)
            _same(got, ref, with_means)
        # a candidate range through the shared array: the same range of dg_grid_search
        w = W.predator_prey(levels=30, noise_seed=5)
        ref = _run(B, B.dg_grid_search, model, w, mode, True, 4097, 9001)
        got = _run(B, B.dg_grid_search_noalloc, model, w, mode, with_means, 4097, 9001)
        _same(got, ref, with_means)
        B.dg_model_free(model)
    finally:
        B.dg_destroy(ctx)


def test_noalloc_rejects_oversized_plain_grid():
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    torch.cuda.init()
    ctx = B.dg_create(0)
    try:
        model = B.compose_predator_prey(ctx)
        w = W.predator_prey(levels=33)   # 35,937 candidates > 32,768
        with pytest.raises(B.DGError) as e:
            _run(B, B.dg_grid_search_noalloc, model, w, 1, False)
        assert e.value.status == B.DG_E_ARG and "32768" in str(e.value)
        B.dg_model_free(model)
    finally:
        B.dg_destroy(ctx)
