"""GPU parity of the coarse-to-fine grid search (the search-space refinement
of Sec. 4.3, by simulation) against the oracle, round by round."""
import numpy as np
import pytest

from gpu_util import MARGIN, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2110_15425_gb300 import binding as B
    torch.cuda.init()
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


def _refine(ctx, pos, lo, hi, G, R, seed, offset=0.1, weight=0.5):
    import torch
    from paper_2110_15425_gb300 import binding as B
    model = B.compose_predator_prey(ctx, obs_offset=offset, pred_weight=weight)
    try:
        out = torch.zeros(R * 64, dtype=torch.uint8, device="cuda")
        B.dg_grid_refine(model, B.refine_desc(dev(pos), lo, hi, G, R, seed), out)
        return B.refine_rounds(host(out))
    finally:
        B.dg_model_free(model)


def _compare(got, ref, R):
    """Round by round while the oracle's decisions are clear of near-ties:
    boxes and allocations bit for bit, indices equal, values within 1e-5."""
    compared = 0
    for r in range(R):
        assert got["round"][r] == r
        np.testing.assert_array_equal(got["lo"][r], ref["box"][r, :3])
        np.testing.assert_array_equal(got["hi"][r], ref["box"][r, 3:])
        assert abs(got["best_value"][r] - ref["value"][r]) <= 1e-5 * max(1.0, abs(ref["value"][r]))
        if ref["gap"][r] < MARGIN:
            break      # the next box depends on a decision within rounding distance
        assert got["best_index"][r] == ref["best"][r], r
        np.testing.assert_array_equal(got["alloc"][r], ref["alloc"][r])
        assert abs(got["runner_up_gap"][r] - ref["gap"][r]) <= 1e-5 * max(1.0, abs(ref["value"][r]))
        compared += 1
    return compared


@pytest.mark.parametrize("G,R,n_trials,lo,hi", [
    (5, 7, 64, [0, 0, 0], [1, 1, 1]),
    (4, 3, 1, [0, 0, 0], [1, 1, 1]),
    (9, 4, 100, [0.0, 0.1, 0.2], [1.0, 0.9, 3.0]),
    (17, 2, 37, [0, 0, 0], [2, 2, 2]),
    (64, 1, 8, [0, 0, 0], [1, 1, 1]),
])
def test_refine_parity(ctx, orc, G, R, n_trials, lo, hi):
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey(n_trials=n_trials)
    got = _refine(ctx, w["pos"], lo, hi, G, R, w["seed"])
    ref = orc.pp_refine(w["pos"], lo, hi, G, R, w["seed"])
    assert _compare(got, ref, R) >= 1


def test_refine_noise_free_closed_form(ctx):
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey(n_trials=16)
    for G in (5, 9):
        got = _refine(ctx, w["pos"], [0, 0, 0], [1, 1, 1], G, 6, w["seed"], offset=1e30)
        assert np.all(got["best_index"] == 0) and np.all(got["alloc"] == 0)
        for r in range(6):
            assert np.all(got["hi"][r] == np.float32((1.0 / (G - 1)) ** r))


def test_refine_round_zero_equals_full_grid(ctx):
    """30 points on [0, 1] are the levels l/29: round 0 is the full grid search."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey()
    got = _refine(ctx, w["pos"], [0, 0, 0], [1, 1, 1], 30, 1, w["seed"])
    model = B.compose_predator_prey(ctx, obs_offset=w["obs_offset"], pred_weight=w["pred_weight"])
    try:
        res = torch.zeros(3, dtype=torch.float64, device="cuda")
        B.dg_grid_search(model, B.grid_desc([dev(l) for l in w["levels"]], dev(w["pos"]),
                                            w["seed"]), res, None)
        r = host(res)
    finally:
        B.dg_model_free(model)
    assert int(r[:1].view(np.int64)[0]) == got["best_index"][0]
    assert r[1] == got["best_value"][0] and r[2] == got["runner_up_gap"][0]


def test_refine_rejects_bad_arguments(ctx):
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey(n_trials=4)
    model = B.compose_predator_prey(ctx)
    out = torch.zeros(64 * 8, dtype=torch.uint8, device="cuda")
    pos = dev(w["pos"])
    try:
        for G, R, lo, hi in ((3, 2, [0] * 3, [1] * 3), (65, 1, [0] * 3, [1] * 3),
                             (5, 2, [0, 1, 0], [1, 0, 1]), (5, 2, [0, float("nan"), 0], [1] * 3),
                             (64, 20000, [0] * 3, [1] * 3), (5, 0, [0] * 3, [1] * 3)):
            with pytest.raises(B.DGError):
                B.dg_grid_refine(model, B.refine_desc(pos, lo, hi, G, R, 1), out)
    finally:
        B.dg_model_free(model)


@pytest.mark.parametrize("G,R,n_trials", [(5, 7, 64), (4, 3, 1), (9, 4, 100), (20, 2, 33)])
def test_refine_cluster_form_equals_launch_per_round(ctx, monkeypatch, G, R, n_trials):
    """The one-cluster search and the launch-per-round search agree bit for bit."""
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey(n_trials=n_trials)
    monkeypatch.setenv("DG_REFINE_FUSED", "0")
    a = _refine(ctx, w["pos"], [0, 0.1, 0], [1, 0.9, 2], G, R, w["seed"])
    monkeypatch.setenv("DG_REFINE_FUSED", "1")
    b = _refine(ctx, w["pos"], [0, 0.1, 0], [1, 0.9, 2], G, R, w["seed"])
    assert a.tobytes() == b.tobytes()
