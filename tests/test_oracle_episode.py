"""Pins of the oracle's time-stepped predator-prey episodes (Sec. 2.1: the
search over attention allocations is repeated at every time step until the
prey or the player is caught)."""
import numpy as np

from paper_2110_15425_gb300 import workloads as W


def test_first_step_is_the_grid_search(orc, threads):
    """Episode 0, step 0 simulates every allocation on perceptions of the
    start positions with the grid search's own noise streams."""
    w = W.predator_prey_episodes(n_episodes=1, levels=6, n_trials=8)
    r = orc.pp_episodes(w["start"], w["levels"], w["n_trials"], 1, w["seed"])
    pos = np.repeat(w["start"][:1], w["n_trials"], axis=0)
    means = orc.pp_means(pos, w["levels"], w["seed"], threads=threads)
    b, _, g = orc.argmax(means)
    assert r["best"][0, 0] == b and r["gap"][0, 0] == g


def _unit(v):
    n = np.hypot(v[0], v[1])
    return v / n if n > 0 else np.zeros(2)


def test_noise_free_moves_closed_form():
    """Without perception noise every allocation sees the true positions, the
    cheapest (index 0) wins, and the moves are pursuit/evasion unit steps from
    the positions at the start of each step."""
    import oracle as orc
    w = W.predator_prey_episodes(n_episodes=6, levels=5, n_trials=3, max_steps=12)
    sp = w["speed"]
    r = orc.pp_episodes(w["start"], w["levels"], 3, 12, w["seed"], obs_offset=1e30,
                        speed=sp, radius=w["radius"])
    for e in range(6):
        S = w["start"][e].astype(np.float32)
        for t in range(int(r["steps"][e])):
            P, D, Y = S[0:2].astype(np.float64), S[2:4].astype(np.float64), S[4:6].astype(np.float64)
            act = _unit(_unit(Y - P) - 0.5 * _unit(D - P))
            N = np.concatenate([P + sp[0] * act, D + sp[1] * _unit(P - D),
                                Y + sp[2] * _unit(Y - P)]).astype(np.float32)
            np.testing.assert_array_equal(r["pos"][e, t], N)
            assert r["best"][e, t] == 0
            S = N
        dy = np.hypot(*(S[0:2].astype(np.float64) - S[4:6]))
        dd = np.hypot(*(S[0:2].astype(np.float64) - S[2:4]))
        expect = 1 if dy <= 1.0 else (-1 if dd <= 1.0 else 0)
        assert r["outcome"][e] == expect
        assert expect != 0 or r["steps"][e] == 12
        np.testing.assert_array_equal(r["final"][e], S)


def test_capture_rules():
    import oracle as orc
    lv = [np.zeros(1, np.float32)] * 3
    # the prey is caught in the first step: P -> (1, 0), Y -> (1.7, 0)
    start = np.array([[0, 0, -100, 0, 1.2, 0]], np.float32)
    r = orc.pp_episodes(start, lv, 1, 5, 1, obs_offset=1e30)
    assert r["outcome"][0] == 1 and r["steps"][0] == 1
    np.testing.assert_allclose(r["final"][0], [1, 0, -99.4, 0, 1.7, 0], rtol=1e-6, atol=1e-6)
    # a fast predator catches the player in the first step
    start = np.array([[0, 0, 1.2, 0, 0, 100]], np.float32)
    r = orc.pp_episodes(start, lv, 1, 5, 1, obs_offset=1e30, speed=(1.0, 1.5, 0.5))
    assert r["outcome"][0] == -1 and r["steps"][0] == 1
    # both at once: the prey counts first
    start = np.array([[0, 0, 1.2, 0, 0, 1.2]], np.float32)
    r = orc.pp_episodes(start, lv, 1, 5, 1, obs_offset=1e30, speed=(1.0, 1.5, 0.1))
    assert r["outcome"][0] == 1
    # nothing within reach: timeout after max_steps
    start = np.array([[0, 0, -100, 0, 100, 0]], np.float32)
    r = orc.pp_episodes(start, lv, 1, 4, 1, obs_offset=1e30)
    assert r["outcome"][0] == 0 and r["steps"][0] == 4 and np.all(r["best"][0] == 0)


def test_episodes_are_independent_streams(orc):
    """An episode's result depends only on its id and start, not on which
    other episodes run beside it."""
    w = W.predator_prey_episodes(n_episodes=4, levels=4, n_trials=4, max_steps=30)
    a = orc.pp_episodes(w["start"], w["levels"], 4, 30, w["seed"])
    b = orc.pp_episodes(w["start"][2:3], w["levels"], 4, 30, w["seed"], episode_ids=[2])
    assert a["outcome"][2] == b["outcome"][0] and a["steps"][2] == b["steps"][0]
    np.testing.assert_array_equal(a["pos"][2], b["pos"][0])
    c = orc.pp_episodes(w["start"][2:3], w["levels"], 4, 30, w["seed"], episode_ids=[3])
    assert not np.array_equal(np.nan_to_num(a["pos"][2]), np.nan_to_num(c["pos"][0]))


def test_episode_noise_layout(orc):
    """Episode e draws its perceptions from Philox blocks 2e and 2e + 1 (normals
    8e .. 8e + 5): step 0's candidate means use streams (trial j, cand c), the
    player's move stream (trial 0, cand 0xFFFFFFFF)."""
    e, n, a = 5, 3, 0.25
    lv = [np.array([a], np.float32)] * 3
    start = np.zeros((e + 1, 6), np.float32)
    start[e] = [1.0, -2.0, 4.0, 3.0, -5.0, 6.0]
    r = orc.pp_episodes(start[e:e + 1], lv, n, 1, 77, episode_ids=[e])
    S = start[e].astype(np.float64)
    sd = 1.0 / (0.1 + np.float64(np.float32(a)))

    def act_of(z):
        ph = S + sd * z
        return _unit(_unit(ph[4:6] - ph[0:2]) - 0.5 * _unit(ph[2:4] - ph[0:2]))
    outs = []
    for j in range(n):
        act = act_of(orc.normals(77, j, 0, 8 * e, 6))
        outs.append(-np.hypot(*(S[0:2] + act - S[4:6])) - 3 * np.float64(np.float32(a)) ** 2)
    assert abs(r["value"][0, 0] - np.mean(outs)) < 1e-12
    act = act_of(orc.normals(77, 0, 0xFFFFFFFF, 8 * e, 6))
    np.testing.assert_allclose(r["pos"][0, 0, 0:2], (S[0:2] + act).astype(np.float32), rtol=0,
                               atol=1e-6)
