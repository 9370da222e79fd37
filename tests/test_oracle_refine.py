"""Pins of the oracle's coarse-to-fine grid search (the search-space
refinement of Sec. 4.3, by simulation)."""
import numpy as np

from paper_2110_15425_gb300 import workloads as W


def test_round_zero_is_the_full_grid(orc, threads):
    """G = 30 points on [0, 1] are the levels l/29 of the full grid search, and
    round 0 draws the full search's noise streams."""
    w = W.predator_prey(n_trials=6)
    r = orc.pp_refine(w["pos"], [0, 0, 0], [1, 1, 1], 30, 1, w["seed"])
    means = orc.pp_means(w["pos"], w["levels"], w["seed"], threads=threads)
    b, bv, g = orc.argmax(means)
    assert (r["best"][0], r["value"][0], r["gap"][0]) == (b, bv, g)
    assert np.array_equal(r["box"][0], np.array([0, 0, 0, 1, 1, 1], np.float32))


def test_noise_free_box_closed_form():
    """Without perception noise the reward does not depend on the allocation,
    so the cheapest point (all zeros) wins every round; the interval around it
    is clipped at 0, so the box [0, hi] shrinks as hi_r = (1 / (G - 1))^r."""
    import oracle as orc
    w = W.predator_prey(n_trials=5)
    for G in (5, 9):
        r = orc.pp_refine(w["pos"], [0, 0, 0], [1, 1, 1], G, 6, w["seed"], obs_offset=1e30)
        assert np.all(r["best"] == 0) and np.all(r["alloc"] == 0)
        for k in range(6):
            assert np.all(r["box"][k, :3] == 0)
            np.testing.assert_array_equal(r["box"][k, 3:], np.float32((1.0 / (G - 1)) ** k))


def _reward(pos, weight=0.5):
    """Mean of -|P + act - Y| with exact perception (numpy restatement)."""
    P, D, Y = pos[:, 0:2].astype(np.float64), pos[:, 2:4].astype(np.float64), pos[:, 4:6].astype(np.float64)

    def unit(v):
        n = np.linalg.norm(v, axis=1, keepdims=True)
        return np.where(n > 0, v / np.where(n > 0, n, 1), 0)
    act = unit(unit(Y - P) - weight * unit(D - P))
    return float(np.mean(-np.linalg.norm(P + act - Y, axis=1)))


def test_noise_free_interior_optimum():
    """On [-0.5, 0.7]^3 the noise-free objective reward - |a|^2 peaks at a = 0,
    strictly inside the domain: every round's value is the exact reward minus
    the cost of its best point, and the best point closes in on 0 within one
    grid spacing per round."""
    import oracle as orc
    w = W.predator_prey(n_trials=7)
    G, R = 5, 8
    r = orc.pp_refine(w["pos"], [-0.5] * 3, [0.7] * 3, G, R, w["seed"], obs_offset=1e30)
    rew = _reward(w["pos"])
    for k in range(R):
        a = r["alloc"][k].astype(np.float64)
        assert abs(r["value"][k] - (rew - np.sum(a * a))) < 1e-12
        spacing = (r["box"][k, 3:].astype(np.float64) - r["box"][k, :3]) / (G - 1)
        # 0 lies in the box, so the nearest grid point is within half a spacing
        assert np.all(np.abs(a) <= spacing / 2 + 1e-7)
        assert np.all((r["box"][k, :3] <= 0) & (r["box"][k, 3:] >= 0))
    assert np.all(np.abs(r["alloc"][-1]) < 1.2 / 2 ** R)


def test_noisy_invariants():
    import oracle as orc
    w = W.predator_prey(n_trials=16)
    lo, hi = np.array([0.0, 0.1, 0.2], np.float32), np.array([1.0, 0.9, 3.0], np.float32)
    for G in (4, 5, 7):
        R = 6
        r = orc.pp_refine(w["pos"], lo, hi, G, R, w["seed"])
        for k in range(R):
            blo, bhi = r["box"][k, :3], r["box"][k, 3:]
            assert np.all(blo >= lo) and np.all(bhi <= hi) and np.all(blo <= bhi)
            b = int(r["best"][k])
            l = np.array([b // (G * G), (b // G) % G, b % G])
            lev = (blo.astype(np.float64) + (bhi.astype(np.float64) - blo) * l / (G - 1))
            np.testing.assert_array_equal(r["alloc"][k], lev.astype(np.float32))
            if k + 1 < R:
                nlo, nhi = r["box"][k + 1, :3], r["box"][k + 1, 3:]
                assert np.all((nlo <= r["alloc"][k]) & (r["alloc"][k] <= nhi))
                width, nwidth = bhi.astype(np.float64) - blo, nhi.astype(np.float64) - nlo
                # endpoints are rounded to FP32: allow two ulps of the largest endpoint
                assert np.all(nwidth <= width * 2 / (G - 1) + 2 * np.spacing(np.float32(3.0)))


def test_rounds_draw_their_own_noise_streams():
    """Round r simulates candidate c on noise stream r G^3 + c: with a
    degenerate domain (every level equal) the rounds evaluate the same
    allocation, and each round's best mean is the average of that stream's
    single-trial outcomes."""
    import oracle as orc
    w = W.predator_prey(n_trials=4)
    G, R = 4, 3
    r = orc.pp_refine(w["pos"], [0.5] * 3, [0.5] * 3, G, R, w["seed"])
    for k in range(R):
        c = int(r["best"][k])
        outs = [orc.pp_outcome(w["pos"][j], [0.5] * 3, w["seed"], j, k * G ** 3 + c)[0]
                for j in range(4)]
        assert abs(r["value"][k] - np.mean(outs)) < 1e-12
    assert len(set(r["value"].tolist())) == R
