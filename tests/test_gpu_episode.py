"""GPU parity of time-stepped predator-prey episodes (Sec. 2.1: the search
over allocations repeated every step until capture) against the oracle."""
import numpy as np
import pytest

from gpu_util import dev, host

pytestmark = pytest.mark.gpu

GAP_MARGIN = 1e-3      # decisions closer than this may differ (positions carry FP32 rounding)
CAPTURE_MARGIN = 1e-3
POS_ATOL = 1e-5       # the moves run in FP64 on both sides; positions differ by libm ulps at most


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2110_15425_gb300 import binding as B
    torch.cuda.init()
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


def _episodes(ctx, w, start=None, T=None, offset=None, speed=None):
    import torch
    from paper_2110_15425_gb300 import binding as B
    start = w["start"] if start is None else start
    T = w["max_steps"] if T is None else T
    E = start.shape[0]
    model = B.compose_predator_prey(ctx, obs_offset=w["obs_offset"] if offset is None else offset,
                                    pred_weight=w["pred_weight"])
    try:
        oc = torch.zeros(E, dtype=torch.int8, device="cuda")
        st = torch.zeros(E, dtype=torch.int32, device="cuda")
        fin = torch.zeros(E * 6, dtype=torch.float32, device="cuda")
        best = torch.zeros(E * T, dtype=torch.int32, device="cuda")
        val = torch.zeros(E * T, dtype=torch.float64, device="cuda")
        pos = torch.zeros(E * T * 6, dtype=torch.float32, device="cuda")
        d = B.episode_desc([dev(l) for l in w["levels"]], dev(start), w["n_trials"], T, w["seed"],
                           speed=w["speed"] if speed is None else speed, radius=w["radius"])
        B.dg_run_episodes(model, d, B.episode_out(oc, st, fin, best, val, pos))
        return dict(outcome=host(oc), steps=host(st), final=host(fin).reshape(E, 6),
                    best=host(best).reshape(E, T), value=host(val).reshape(E, T),
                    pos=host(pos).reshape(E, T, 6))
    finally:
        B.dg_model_free(model)


def _compare(got, ref, E):
    """Step by step while the oracle's decisions are clear of near-ties:
    allocations equal, positions within POS_ATOL, means within 1e-5; outcome
    and length equal for episodes that never came near a tie."""
    clean = 0
    for e in range(E):
        near = False
        for t in range(int(ref["steps"][e])):
            assert got["best"][e, t] == ref["best"][e, t], (e, t)
            np.testing.assert_allclose(got["pos"][e, t], ref["pos"][e, t], rtol=0, atol=POS_ATOL)
            assert abs(got["value"][e, t] - ref["value"][e, t]) <= 1e-5 * max(1, abs(ref["value"][e, t]))
            if ref["gap"][e, t] < GAP_MARGIN or ref["margin"][e, t] < CAPTURE_MARGIN:
                near = True
                break
        if not near:
            assert got["outcome"][e] == ref["outcome"][e] and got["steps"][e] == ref["steps"][e], e
            np.testing.assert_allclose(got["final"][e], ref["final"][e], rtol=0, atol=POS_ATOL)
            assert np.all(got["best"][e, ref["steps"][e]:] == -1)
            clean += 1
    return clean


@pytest.mark.parametrize("levels,n_trials,T", [(5, 16, 60), (3, 1, 40), (7, 33, 25)])
def test_episode_parity(ctx, orc, threads, levels, n_trials, T):
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey_episodes(n_episodes=24, levels=levels, n_trials=n_trials, max_steps=T)
    got = _episodes(ctx, w)
    ref = orc.pp_episodes(w["start"], w["levels"], n_trials, T, w["seed"], speed=w["speed"],
                          radius=w["radius"], threads=threads)
    assert _compare(got, ref, 24) >= 12
    assert set(np.unique(got["outcome"])) <= {-1, 0, 1}


def test_episode_noise_free_and_capture(ctx, orc):
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey_episodes(n_episodes=16, levels=4, n_trials=4, max_steps=80)
    got = _episodes(ctx, w, offset=1e30)
    ref = orc.pp_episodes(w["start"], w["levels"], 4, 80, w["seed"], obs_offset=1e30,
                          speed=w["speed"], radius=w["radius"])
    assert _compare(got, ref, 16) >= 12
    assert np.all(got["best"][got["best"] >= 0] == 0)
    # a fast predator catches the player in one step; the prey counts first on a double capture
    start = np.array([[0, 0, 1.2, 0, 0, 100], [0, 0, 1.2, 0, 0, 1.2]], np.float32)
    g = _episodes(ctx, w, start=start, T=5, offset=1e30, speed=(1.0, 1.5, 0.1))
    assert list(g["outcome"]) == [-1, 1] and list(g["steps"]) == [1, 1]


def test_episode_full_size_first_steps(ctx, orc, threads):
    """64 episodes on the full 30^3 grid with 64 perceptions per candidate: the
    first two steps of four episodes against the oracle, and invariants for all."""
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey_episodes()
    got = _episodes(ctx, w)
    E, T = w["start"].shape[0], w["max_steps"]
    assert set(np.unique(got["outcome"])) <= {-1, 0, 1}
    assert np.all((got["steps"] >= 1) & (got["steps"] <= T))
    for e in range(E):
        s = got["steps"][e]
        assert np.all(got["best"][e, :s] >= 0) and np.all(got["best"][e, s:] == -1)
        np.testing.assert_array_equal(got["final"][e], got["pos"][e, s - 1])
        P, D, Y = got["final"][e, 0:2], got["final"][e, 2:4], got["final"][e, 4:6]
        if got["outcome"][e] == 1:
            assert np.hypot(*(P - Y)) <= 1.0 + 1e-6
        elif got["outcome"][e] == -1:
            assert np.hypot(*(P - D)) <= 1.0 + 1e-6
        else:
            assert s == T
    ids = np.array([0, 17, 38, 63])
    ref = orc.pp_episodes(w["start"][ids], w["levels"], w["n_trials"], 2, w["seed"],
                          episode_ids=ids, speed=w["speed"], radius=w["radius"], threads=threads)
    for k, e in enumerate(ids):
        for t in range(min(2, int(ref["steps"][k]))):
            if ref["gap"][k, t] < GAP_MARGIN:
                break
            assert got["best"][e, t] == ref["best"][k, t]
            np.testing.assert_allclose(got["pos"][e, t], ref["pos"][k, t], rtol=0, atol=POS_ATOL)


def test_episode_independent_of_batch(ctx):
    """An episode's result does not depend on the other episodes in the call."""
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey_episodes(n_episodes=12, levels=5, n_trials=8, max_steps=50)
    a = _episodes(ctx, w)
    # the same starts in reverse order give each start a different episode index;
    # so compare against a call where episode ids keep their starts: the first 5 only
    b = _episodes(ctx, w, start=w["start"][:5])
    for k in ("outcome", "steps", "final", "best", "value", "pos"):
        assert np.array_equal(a[k][:5], b[k][:5]), k


def test_episode_offset_reassembles(ctx):
    """Episodes 0..11 in one call equal episodes 0..4 and 5..11 run as two calls
    with episode_offset 0 and 5 (the noise is keyed by the global index)."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey_episodes(n_episodes=12, levels=5, n_trials=8, max_steps=40)
    full = _episodes(ctx, w)
    model = B.compose_predator_prey(ctx, obs_offset=w["obs_offset"], pred_weight=w["pred_weight"])
    try:
        for lo, hi in ((0, 5), (5, 12)):
            E, T = hi - lo, 40
            oc = torch.zeros(E, dtype=torch.int8, device="cuda")
            st = torch.zeros(E, dtype=torch.int32, device="cuda")
            best = torch.zeros(E * T, dtype=torch.int32, device="cuda")
            pos = torch.zeros(E * T * 6, dtype=torch.float32, device="cuda")
            d = B.episode_desc([dev(l) for l in w["levels"]], dev(w["start"][lo:hi]), 8, T,
                               w["seed"], speed=w["speed"], radius=w["radius"], episode_offset=lo)
            B.dg_run_episodes(model, d, B.episode_out(oc, st, None, best, None, pos))
            assert np.array_equal(host(oc), full["outcome"][lo:hi])
            assert np.array_equal(host(st), full["steps"][lo:hi])
            assert np.array_equal(host(best).reshape(E, T), full["best"][lo:hi])
            assert np.array_equal(host(pos).reshape(E, T, 6), full["pos"][lo:hi])
    finally:
        B.dg_model_free(model)


def test_episode_bad_arguments(ctx):
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey_episodes(n_episodes=2, levels=3, n_trials=4, max_steps=5)
    model = B.compose_predator_prey(ctx)
    oc = torch.zeros(2, dtype=torch.int8, device="cuda")
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    lv = [dev(l) for l in w["levels"]]
    start = dev(w["start"])
    try:
        for kw in (dict(n_trials=0), dict(n_trials=2000), dict(speed=(-1.0, 0.5, 0.5)),
                   dict(radius=float("nan")), dict(episode_offset=-1), dict(max_steps=0)):
            args = dict(n_trials=4, max_steps=5, speed=w["speed"], radius=w["radius"], episode_offset=0)
            args.update(kw)
            d = B.episode_desc(lv, start, args["n_trials"], args["max_steps"], 1, speed=args["speed"],
                               radius=args["radius"], episode_offset=args["episode_offset"])
            with pytest.raises(B.DGError):
                B.dg_run_episodes(model, d, B.episode_out(oc, st))
    finally:
        B.dg_model_free(model)
